// Backward JTFS kernels (Sec. 5: reverse-ordered adjoints of the forward operators), FP32
// on CUDA cores.  Only the first-order scalogram U1 is checkpointed by the forward; the
// backward recomputes x-hat, U1-hat, Y_alpha and Z, and the first-order coefficients z.
//
//   k_uh_from_u1       : U1-hat = FFT of every checkpointed U1 row
//   k_joint_bwd_simt   : per (alpha, 32-column chunk, signal): for every channel c,
//                        Z = W_c Y, g|Z| = adjoint of phi_T x phi_F pooling applied to g_S2,
//                        gZ = g|Z| Z / |Z| (0 at Z = 0), gY += W_c^H gZ
//   k_gy_spectra       : DFT of every gY row, in place (G rows of one rate per CTA)
//   k_second_order_bwd : per (lambda', signal): sum over alpha of the adjoint of the
//                        fold / psi_alpha product on those spectra, real part of the inverse
//                        of the row FFT, plus the adjoint of S1's pooling -> g_U1 row
//   k_stage1_bwd       : per (lambda, signal): recompute z, gz = g_U1 z / |z|, FFT -> gF
//   k_gxh              : g_x-hat[k] = sum_lambda psi_lambda[k] gF_lambda[k mod L_lambda], plus
//                        the spectrum of S0's adjoint
//   k_gx               : g_x = Re(inverse DFT of g_x-hat)
#include <mutex>

#include "stages.cuh"

namespace jtfs {
namespace {

__global__ void __launch_bounds__(kFftThreads)
k_uh_from_u1(DevPlan P, const float* __restrict__ u1, float2* __restrict__ uh) {
  extern __shared__ float2 sm[];
  const int lam = blockIdx.x, b = blockIdx.y;
  const Row1 R = P.rows1[lam];
  const float* ub = u1 + (size_t)b * P.u1_len + R.off_u;
  for (int m = threadIdx.x; m < R.L; m += blockDim.x)
    sm[fft_pos(bitrev(m, R.logL), R.logL)] = make_float2(ub[m], 0.f);
  __syncthreads();
  fft_dit_rows_r16<-1>(sm, R.logL, 1, twl_for(P, R.logL));
  float2* hb = uh + (size_t)b * P.uh_len + R.off_uh;
  for (int k = threadIdx.x; k < (R.L >> 1); k += blockDim.x) hb[k] = sm[fft_pos(k, R.logL)];
}

// ---------------------------------------------------------------------------------------
constexpr int kJT = 256;
constexpr int kNC = 32;
constexpr int kRPT = 8;

__global__ void __launch_bounds__(kJT)
k_joint_bwd_simt(DevPlan P, const int2* __restrict__ items, const float2* __restrict__ y,
                 const float* __restrict__ gs2, float2* __restrict__ gy) {
  extern __shared__ float4 smraw[];
  const int2 it = items[blockIdx.x];
  const int a = it.x, n0 = it.y, b = blockIdx.y;
  const Rate2 A = P.rates2[a];
  const int n1 = P.n1, nt = P.n_t, K = A.K, l0 = A.lam_min, nfm = P.N_fr - 1;
  float2* sh = reinterpret_cast<float2*>(smraw);        // [N_fr]
  float2* yt = sh + P.N_fr;                              // [K][kNC]
  float2* gz = yt + (size_t)n1 * kNC;                    // [n1][kNC]
  float* g1 = reinterpret_cast<float*>(gz + (size_t)n1 * kNC);  // [n1][n_t]
  float* wt = g1 + (size_t)n1 * nt;                      // [n_t][kNC]
  const float2* ya = y + (size_t)b * P.y_len + A.off_y;
  for (int i = threadIdx.x; i < K * kNC; i += blockDim.x) {
    const int k = i / kNC, col = i % kNC;
    yt[i] = (n0 + col < A.L) ? ya[(size_t)k * A.L + n0 + col] : make_float2(0.f, 0.f);
  }
  for (int i = threadIdx.x; i < nt * kNC; i += blockDim.x) {
    const int t = i / kNC, col = i % kNC;
    const int n = n0 + col;
    wt[i] = (n < A.L) ? __ldg(&P.phiT[(t * P.T - n * A.s) & (P.N - 1)]) * (float)A.s : 0.f;
  }
  const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;
  float2 gacc[kRPT][4];
#pragma unroll
  for (int i = 0; i < kRPT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) gacc[i][j] = make_float2(0.f, 0.f);

  for (int c = 0; c < P.C; ++c) {
    __syncthreads();
    for (int i = threadIdx.x; i < P.N_fr; i += blockDim.x) sh[i] = P.h[(size_t)c * P.N_fr + i];
    const float* g = gs2 + (size_t)b * P.s2_stride + ((size_t)a * P.C + c) * P.n_lo * nt;
    for (int i = threadIdx.x; i < n1 * nt; i += blockDim.x) {
      if (P.average_fr) {
        const int r = i / nt, t = i % nt;
        float s = 0.f;
        for (int lo = 0; lo < P.n_lo; ++lo)
          s += __ldg(&P.phiF[(lo * P.s_F - r) & nfm]) * g[lo * nt + t];
        g1[i] = s;
      } else {
        g1[i] = g[i];
      }
    }
    __syncthreads();
    // Z = W_c Y for the thread's (row, column) outputs
    float2 acc[kRPT][4];
#pragma unroll
    for (int i = 0; i < kRPT; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) {
      const float4 y01 = reinterpret_cast<const float4*>(yt + k * kNC)[tx * 2];
      const float4 y23 = reinterpret_cast<const float4*>(yt + k * kNC)[tx * 2 + 1];
      const float2 yv[4] = {make_float2(y01.x, y01.y), make_float2(y01.z, y01.w),
                            make_float2(y23.x, y23.y), make_float2(y23.z, y23.w)};
      const int kk = k + l0;
#pragma unroll
      for (int i = 0; i < kRPT; ++i) {
        const int r = ty + 32 * i;
        if (r < n1) {
          const float2 hv = sh[(r - kk) & nfm];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x += hv.x * yv[j].x - hv.y * yv[j].y;
            acc[i][j].y += hv.x * yv[j].y + hv.y * yv[j].x;
          }
        }
      }
    }
    // g|Z| = sum_t g1[r][t] w[t][col];  gZ = g|Z| Z / |Z|
#pragma unroll
    for (int i = 0; i < kRPT; ++i) {
      const int r = ty + 32 * i;
      if (r < n1) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int col = tx * 4 + j;
          float ga = 0.f;
          for (int t = 0; t < nt; ++t) ga += g1[r * nt + t] * wt[t * kNC + col];
          const float2 z = acc[i][j];
          const float m = sqrtf(z.x * z.x + z.y * z.y);
          const float f = (m > 0.f) ? ga / m : 0.f;
          gz[r * kNC + col] = make_float2(z.x * f, z.y * f);
        }
      }
    }
    __syncthreads();
    // gY[k][col] += sum_r conj(h_c[(r - k) mod N_fr]) gZ[r][col]
    for (int r = 0; r < n1; ++r) {
      const float4 g01 = reinterpret_cast<const float4*>(gz + r * kNC)[tx * 2];
      const float4 g23 = reinterpret_cast<const float4*>(gz + r * kNC)[tx * 2 + 1];
      const float2 gv[4] = {make_float2(g01.x, g01.y), make_float2(g01.z, g01.w),
                            make_float2(g23.x, g23.y), make_float2(g23.z, g23.w)};
#pragma unroll
      for (int i = 0; i < kRPT; ++i) {
        const int k = ty + 32 * i;
        if (k < K) {
          const float2 hv = sh[(r - k - l0) & nfm];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            gacc[i][j].x += hv.x * gv[j].x + hv.y * gv[j].y;
            gacc[i][j].y += hv.x * gv[j].y - hv.y * gv[j].x;
          }
        }
      }
    }
  }
  float2* go = gy + (size_t)b * P.y_len + A.off_y;
#pragma unroll
  for (int i = 0; i < kRPT; ++i) {
    const int k = ty + 32 * i;
    if (k < K)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int col = tx * 4 + j;
        if (n0 + col < A.L) go[(size_t)k * A.L + n0 + col] = gacc[i][j];
      }
  }
}

// Spectra of the gY rows, in place: G rows of one rate per CTA (the Y producer's row items),
// batched forward FFT (padded radix-16 passes, bit-reversed loads), written back in natural
// order.
__global__ void __launch_bounds__(kRowBound)
k_gy_spectra(DevPlan P, const int4* __restrict__ items, float2* __restrict__ gy) {
  extern __shared__ float2 sm[];
  const int4 it = items[blockIdx.x];
  const int a = it.x, lam0 = it.y, G = it.z, b = blockIdx.y;
  const Rate2 A = P.rates2[a];
  const int L = A.L, logL = A.logL;
  float2* g = gy + (size_t)b * P.y_len + A.off_y + (size_t)(lam0 - A.lam_min) * L;
  const int total = G * L, step = blockDim.x;
  // two samples per 16-byte access where the block's rows start 16-byte aligned (rows hold an
  // even number of samples), else one
  const bool pair = L >= 2 && ((uintptr_t)g & 15) == 0;
  if (pair) {
    // four 16-byte loads in flight per thread before their shared-memory stores
    const float4* g4 = reinterpret_cast<const float4*>(g);
    const int total2 = total >> 1;
    for (int base = threadIdx.x; base < total2; base += 4 * step) {
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i2 = base + q * step;
        v[q] = i2 < total2 ? g4[i2] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = 2 * (base + q * step);
        if (idx < total) {
          const int r0 = (idx >> logL) << logL, k = idx & (L - 1);
          sm[fft_pos(r0 + bitrev(k, logL), logL)] = make_float2(v[q].x, v[q].y);
          sm[fft_pos(r0 + bitrev(k + 1, logL), logL)] = make_float2(v[q].z, v[q].w);
        }
      }
    }
  } else {
    // eight loads in flight per thread before their shared-memory stores
    for (int base = threadIdx.x; base < total; base += 8 * step) {
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int idx = base + q * step;
        v[q] = idx < total ? g[idx] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int idx = base + q * step;
        if (idx < total) sm[fft_pos(((idx >> logL) << logL) + bitrev(idx & (L - 1), logL), logL)] = v[q];
      }
    }
  }
  __syncthreads();
  fft_dit_rows_r16<-1>(sm, logL, G, twl_for(P, logL));
  if (pair) {
    float4* g4 = reinterpret_cast<float4*>(g);
    for (int i2 = threadIdx.x; i2 < total >> 1; i2 += blockDim.x) {
      const float2 a = sm[fft_pos(2 * i2, logL)], c = sm[fft_pos(2 * i2 + 1, logL)];
      g4[i2] = make_float4(a.x, a.y, c.x, c.y);
    }
  } else {
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) g[idx] = sm[fft_pos(idx, logL)];
  }
}

// g_U1 row lambda': sum over rates alpha of the adjoint of psi2 (the gY row's spectrum / Lr
// times psi-hat_alpha on the row's positive bins), then Re of the inverse row DFT, plus S1's
// adjoint.
__global__ void __launch_bounds__(256, 3)   // launched with 256 threads; three blocks per SM
k_second_order_bwd(DevPlan P, const float2* __restrict__ gys, const float* __restrict__ gs1,
                   float* __restrict__ gu1) {
  extern __shared__ float2 sm[];
  const int lam = blockIdx.x, b = blockIdx.y;
  const Row1 R = P.rows1[lam];
  const int half = R.L >> 1;
  float2* tmp = sm;                // [L] padded
  const float invLr = 1.f / (float)R.L;
  const float* g1 = gs1 ? gs1 + ((size_t)b * P.n1 + lam) * P.n_t : nullptr;
  // guh[k] for k <= half, built in registers per bin and stored bit-reversed; g_U1 is the real
  // part of its inverse DFT.  Two terms:
  //  - the rates' adjoint: the gY row spectra / Lr times psi-hat_alpha on bins 0 < k < half;
  //  - S1's adjoint g[m] = s sum_t phi_T[t T - m s] g_S1[t], whose length-L DFT is
  //    G[k mod n_t] sum_r phi-hat[k + r L] (the spikes of g_S1 sit tau = T / s apart and
  //    phi_T at stride s aliases phi-hat): nonzero only where phi-hat is, taken one-sided
  //    (bins 0 and L / 2 once, the others twice), with phi-hat on the bins phi_T is built from.
  for (int k = threadIdx.x; k < R.L; k += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    if (k >= 1 && k < half) {
      // the rates in groups of eight whose loads are in flight together, summed in
      // increasing alpha (a rate outside its support adds 0 * 0)
      for (int a0 = 0; a0 < P.n2; a0 += 8) {
        float2 v[8];
        float f[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int a = a0 + q;
          v[q] = make_float2(0.f, 0.f);
          f[q] = 0.f;
          if (a < P.n2) {
            const Rate2 A = P.rates2[a];
            if (A.s != 0 && lam >= A.lam_min && k < A.k2e) {
              v[q] = gys[(size_t)b * P.y_len + A.off_y + (size_t)(lam - A.lam_min) * A.L +
                         (k & (A.L - 1))];
              f[q] = __ldg(&P.psi2[(size_t)a * P.K2max + k]) * invLr;
            }
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          acc.x += v[q].x * f[q];
          acc.y += v[q].y * f[q];
        }
      }
    }
    if (g1 && k <= half) {
      // signed representatives k + r L of the N-grid bins: r >= 0, then r < 0
      // (|k + r L| = |r| L - k, below the Nyquist bin, which the first loop holds)
      float ph = 0.f;
      const int qneg = min(P.phiT_kmax, (P.N >> 1) - 1);
      for (int q = k; q <= P.phiT_kmax; q += R.L) ph += __ldg(&P.phiThat[q]);
      for (int q = R.L - k; q <= qneg; q += R.L) ph += __ldg(&P.phiThat[q]);
      if (ph != 0.f) {
        const int f = k & (P.n_t - 1);
        float2 G = make_float2(0.f, 0.f);
        for (int t = 0; t < P.n_t; ++t) {   // G[f] = sum_t g_S1[t] exp(-2 pi i f t / n_t)
          float sn, cs;
          sincospif(2.f * (float)((f * t) & (P.n_t - 1)) / (float)P.n_t, &sn, &cs);
          G.x += g1[t] * cs;
          G.y -= g1[t] * sn;
        }
        const float c = ((k == 0 || k == half) ? 1.f : 2.f) * invLr * ph;
        acc.x += c * G.x;
        acc.y += c * G.y;
      }
    }
    tmp[fft_pos(bitrev(k, R.logL), R.logL)] = acc;
  }
  __syncthreads();
  fft_dit_rows_r16<+1>(tmp, R.logL, 1, twl_for(P, R.logL));
  float* out = gu1 + (size_t)b * P.u1_len + R.off_u;
  for (int m = threadIdx.x; m < R.L; m += blockDim.x) out[m] = tmp[fft_pos(m, R.logL)].x;
}

__global__ void __launch_bounds__(kRowLaunch, 3)   // three 256-thread blocks per SM
k_stage1_bwd(DevPlan P, const float2* __restrict__ xh, const float* __restrict__ gu1,
             float2* __restrict__ gf) {
  extern __shared__ float2 sm[];
  const int lam = blockIdx.x, b = blockIdx.y;
  const Row1 R = P.rows1[lam];
  fold_first_order(P, R, xh + (size_t)b * (P.N >> 1), sm);
  __syncthreads();
  fft_dit_rows_r16<+1>(sm, R.logL, 1, twl_for(P, R.logL));
  // gz = g_U1 z / |z| (0 at z = 0), stored bit-reversed for the forward FFT: every thread
  // handles the pairs (m, bitrev(m)) with m <= bitrev(m), so the permutation is in place
  const float* g = gu1 + (size_t)b * P.u1_len + R.off_u;
  for (int m = threadIdx.x; m < R.L; m += blockDim.x) {
    const int r = bitrev(m, R.logL);
    if (m > r) continue;
    const float2 zm = sm[fft_pos(m, R.logL)], zr = sm[fft_pos(r, R.logL)];   // N * z
    const float am = hypotf(zm.x, zm.y), ar = hypotf(zr.x, zr.y);
    const float fm = (am > 0.f) ? g[m] / am : 0.f, fr = (ar > 0.f) ? g[r] / ar : 0.f;
    sm[fft_pos(r, R.logL)] = make_float2(zm.x * fm, zm.y * fm);
    sm[fft_pos(m, R.logL)] = make_float2(zr.x * fr, zr.y * fr);
  }
  __syncthreads();
  fft_dit_rows_r16<-1>(sm, R.logL, 1, twl_for(P, R.logL));
  const float invN = 1.f / (float)P.N;
  float2* out = gf + (size_t)b * P.u1_len + R.off_u;
  for (int k = threadIdx.x; k < R.L; k += blockDim.x) {
    const float2 v = sm[fft_pos(k, R.logL)];
    out[k] = make_float2(v.x * invN, v.y * invN);
  }
}

// S0's adjoint sum_t phi_T[(tT - n) mod N] g_S0[t] has the length-N DFT
// DFT(g_S0)[k mod n_t] phi-hat[k] (spikes T apart), nonzero for k <= phiT_kmax: it is added
// to those bins of the one-sided g_x spectrum (bin 0 once, the others twice, / N).  When
// phi-hat reaches the Nyquist bin (T <= 2), k_gx adds it in the time domain instead.
__global__ void k_gxh(DevPlan P, const float2* __restrict__ gf, const float* __restrict__ gs0,
                      float2* __restrict__ gxh) {
  const int b = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int half = P.N >> 1;
  const int2 rng = P.gx_lam[blockIdx.x];
  float2 acc = make_float2(0.f, 0.f);
  if (k < half) {
    const float2* gb = gf + (size_t)b * P.u1_len;
    for (int lam = rng.x; lam < rng.y; ++lam) {
      const Row1 R = P.rows1[lam];
      const int i = k - R.ks;
      if (i >= 0 && i < R.kl) {
        const float f = __ldg(&P.psi1[R.off_v + i]);
        const float2 v = gb[R.off_u + (k & (R.L - 1))];
        acc.x += f * v.x;
        acc.y += f * v.y;
      }
    }
    if (gs0 && k <= P.phiT_kmax && P.phiT_kmax < half) {
      const float* g0 = gs0 + (size_t)b * P.n_t;
      const int f = k & (P.n_t - 1);
      float2 G = make_float2(0.f, 0.f);
      for (int t = 0; t < P.n_t; ++t) {
        float sn, cs;
        sincospif(2.f * (float)((f * t) & (P.n_t - 1)) / (float)P.n_t, &sn, &cs);
        G.x += g0[t] * cs;
        G.y -= g0[t] * sn;
      }
      const float c = (k == 0 ? 1.f : 2.f) * __ldg(&P.phiThat[k]) / (float)P.N;
      acc.x += c * G.x;
      acc.y += c * G.y;
    }
    gxh[(size_t)b * half + k] = acc;
  }
}

// g_x[r + D m] = Re(sum_k' e^{2 pi i k' m / M} sum_q H[k' + q M] e^{2 pi i (k' + q M) r / N})
// (S0's adjoint is already in H unless phi-hat reaches the Nyquist bin)
__global__ void __launch_bounds__(kFftThreads, 2)   // two 512-thread blocks per SM
k_gx(DevPlan P, const float2* __restrict__ gxh, const float* __restrict__ gs0, float* __restrict__ gx) {
  extern __shared__ float2 sm[];
  const int r = blockIdx.x, b = blockIdx.y;
  const int half = P.N >> 1;
  const int step = P.TW / P.N;
  const float2* H = gxh + (size_t)b * half;
  for (int kp = threadIdx.x; kp < P.M; kp += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int k = kp; k < half; k += P.M) {
      const float2 v = H[k];
      const int idx = (int)(((long long)k * r) & (P.N - 1)) * step;
      float2 w = __ldg(&P.tw[idx]);
      w.y = -w.y;
      acc.x += v.x * w.x - v.y * w.y;
      acc.y += v.x * w.y + v.y * w.x;
    }
    sm[fft_pos(bitrev(kp, P.logM), P.logM)] = acc;
  }
  __syncthreads();
  fft_dit_rows_r16<+1>(sm, P.logM, 1, twl_for(P, P.logM));
  const float* g0 = (gs0 && P.phiT_kmax >= half) ? gs0 + (size_t)b * P.n_t : nullptr;
  float* out = gx + (size_t)b * P.N;
  for (int m = threadIdx.x; m < P.M; m += blockDim.x) {
    const int n = r + P.D * m;
    float v = sm[fft_pos(m, P.logM)].x;
    if (g0)
      for (int t = 0; t < P.n_t; ++t) v += __ldg(&P.phiT[(t * P.T - n) & (P.N - 1)]) * g0[t];
    out[n] = v;
  }
}

// Time scattering (Scattering1D) backward of the second order: Y_alpha rows recomputed in
// shared memory as in the forward, then gY = g_|Y| Y / |Y| (0 where Y = 0) with
// g_|Y|[m] = sum_t s_alpha phi_T[(t T - m s_alpha) mod N] g_S2t[t], written in the layout of the
// transform's gY so that the second-order adjoint that follows is shared.
__global__ void __launch_bounds__(kRowBound)
k_scat1d_bwd_rows(DevPlan P, const int4* __restrict__ items, const float2* __restrict__ uh,
                  const float* __restrict__ gs2t, float2* __restrict__ gy) {
  extern __shared__ float2 sm[];
  __shared__ int s_off[kMaxRowsPerItem], s_kend[kMaxRowsPerItem];
  __shared__ float s_inv[kMaxRowsPerItem];
  const int4 it = items[blockIdx.x];
  const int a = it.x, lam0 = it.y, G = it.z, b = blockIdx.y;
  const Rate2 A = P.rates2[a];
  const int L = A.L, logL = A.logL, nt = P.n_t;
  second_order_rows_ifft(P, A, a, lam0, G, uh + (size_t)b * P.uh_len, sm, s_off, s_kend, s_inv);
  __syncthreads();
  const float* g = gs2t + (((size_t)b * P.n2 + a) * P.n1 + lam0) * nt;
  float2* out = gy + (size_t)b * P.y_len + A.off_y + (size_t)(lam0 - A.lam_min) * L;
  for (int idx = threadIdx.x; idx < G * L; idx += blockDim.x) {
    const int r = idx >> logL, m = idx & (L - 1);
    float ga = 0.f;
    for (int t = 0; t < nt; ++t)
      ga = fmaf(__ldg(&P.phiT[((long long)t * P.T - (long long)m * A.s) & (P.N - 1)]),
                __ldg(&g[r * nt + t]), ga);
    const float2 v = sm[fft_pos(idx, logL)];
    const float mag = sqrtf(v.x * v.x + v.y * v.y);
    const float sc = mag > 0.f ? ga * (float)A.s / mag : 0.f;
    out[idx] = make_float2(v.x * sc, v.y * sc);
  }
}

// cudaFuncSetAttribute acts on the current device only, so the raised shared-memory limits
// are recorded per device (the plan's device is current in every call that launches).
std::mutex g_attrs_mu;
bool g_attrs_set[256] = {};

jtfs_status set_attrs(const jtfs_plan* p) {
  if (p->device < 0 || p->device >= 256) {
    set_error("device ordinal out of range");
    return JTFS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_attrs_mu);
  if (g_attrs_set[p->device]) return JTFS_OK;
  const int big = 227 * 1024;
  const void* fns[] = {(const void*)k_uh_from_u1, (const void*)k_joint_bwd_simt,
                       (const void*)k_second_order_bwd, (const void*)k_stage1_bwd,
                       (const void*)k_gx, (const void*)k_xfft_sub};
  for (const void* f : fns) {
    jtfs_status st = cuda_check(
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big), "attr");
    if (st != JTFS_OK) return st;
  }
  // the row producer holds at most 2^14 complex samples (padded one per 16) next to its
  // static row tables
  for (const void* f : {(const void*)k_second_order_rows<0>, (const void*)k_second_order_rows<1>,
                        (const void*)k_gy_spectra, (const void*)k_scat1d_bwd_rows}) {
    jtfs_status st = cuda_check(
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 140 * 1024), "attr");
    if (st != JTFS_OK) return st;
  }
  g_attrs_set[p->device] = true;
  return JTFS_OK;
}

}  // namespace

size_t joint_bwd_smem(const jtfs_plan* p) {
  return (size_t)p->N_fr * 8 + 2 * (size_t)p->n1 * kNC * 8 + (size_t)p->n1 * p->n_t * 4 +
         (size_t)p->n_t * kNC * 4;
}

bool backward_reuses_forward(const jtfs_plan* p) {
  // the forward's BF16 Y planes are the backward's operands (not for TF32, whose forward
  // writes FP32 planes)
  return p->use_tc && p->use_tcb && p->cfg.precision != JTFS_PREC_TF32;
}

jtfs_status launch_backward(const jtfs_plan* p, const float* x, const float* u1, int B,
                            const float* gs0, const float* gs1, const float* gs2, float* gx,
                            const Workspace& w, cudaStream_t st, bool fused) {
  jtfs_status rc = set_attrs(p);
  if (rc != JTFS_OK) return rc;
  const DevPlan& d = p->dp;
  // fused: x-hat, U1-hat (and the BF16 Y planes) are still in the workspace from the forward
  // of the same call; otherwise recompute them from x and the checkpoint
  const bool reuse_y = fused && backward_reuses_forward(p);
  if (!fused) {
    {
      StageScope sc(p, kStXfft, st, 2);
      k_xfft_sub<<<dim3(d.D, B), kFftThreads, (size_t)d.M * 17 / 2, st>>>(d, x, w.xsub);
      k_xfft_combine<<<dim3((p->N / 2 + 255) / 256, B), 256, 0, st>>>(d, w.xsub, w.xh);
    }
    {
      StageScope sc(p, kStUhFromU1, st, 1);
      k_uh_from_u1<<<dim3(p->n1, B), kFftThreads, (size_t)p->L1max * 17 / 2, st>>>(d, u1, w.uh);
    }
  }
  const size_t n_items = p->items.size() / 2;
  if (gs2 && n_items > 0 && p->use_tcb) {
    if (!reuse_y) {
      StageScope sc(p, kStSecondOrder, st, 1);
      k_second_order_rows<1><<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                              (size_t)p->rows_cap * 17 / 2, st>>>(
          d, reinterpret_cast<const int4*>(p->d_rowitems), w.uh, nullptr,
          (__nv_bfloat16*)w.ybh, (__nv_bfloat16*)w.ybl, B);
    }
    StageScope sc(p, kStJointBwd, st, 0);   // the launcher counts its kernels
    jtfs_status r2 = launch_joint_bwd_tc(p, B, w.ybh, w.ybl, gs2, w.g1, w.gy, st);
    if (r2 != JTFS_OK) return r2;
    if (!p->tcb_fb_items.empty()) {
      // rates beyond the tensor-core backward's lambda' capacity: FP32 Y rows of those rates
      // only, then the CUDA-core backward on them
      k_second_order_rows<0><<<dim3((unsigned)(p->tcb_fb_rowitems.size() / 4), B),
                              p->row_threads, (size_t)p->tcb_fb_cap * 17 / 2, st>>>(
          d, reinterpret_cast<const int4*>(p->d_tcb_fb_rowitems), w.uh, w.y, nullptr, nullptr,
          B);
      k_joint_bwd_simt<<<dim3((unsigned)(p->tcb_fb_items.size() / 2), B), kJT,
                         joint_bwd_smem(p), st>>>(
          d, reinterpret_cast<const int2*>(p->d_tcb_fb_items), w.y, gs2, w.gy);
      p->prof.launches += 2;
    }
  } else if (gs2 && n_items > 0) {
    {
      StageScope sc(p, kStSecondOrder, st, 1);
      k_second_order_rows<0><<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                              (size_t)p->rows_cap * 17 / 2, st>>>(
          d, reinterpret_cast<const int4*>(p->d_rowitems), w.uh, w.y, nullptr, nullptr, B);
    }
    StageScope sc(p, kStJointBwd, st, 1);
    k_joint_bwd_simt<<<dim3((unsigned)n_items, B), kJT, joint_bwd_smem(p), st>>>(
        d, reinterpret_cast<const int2*>(p->d_items), w.y, gs2, w.gy);
  } else if (p->y_len > 0) {
    cudaMemsetAsync(w.gy, 0, (size_t)B * p->y_len * sizeof(float2), st);
  }
  {
    StageScope sc(p, kStSecondOrderBwd, st, 2);
    if (!p->rowitems.empty())
      k_gy_spectra<<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                     (size_t)p->rows_cap * 17 / 2, st>>>(
          d, reinterpret_cast<const int4*>(p->d_rowitems), w.gy);
    k_second_order_bwd<<<dim3(p->n1, B), 256, (size_t)p->L1max * 17 / 2, st>>>(d, w.gy, gs1, w.gu1);
  }
  {
    StageScope sc(p, kStStage1Bwd, st, 1);
    k_stage1_bwd<<<dim3(p->n1, B), kRowLaunch, (size_t)p->L1max * 17 / 2, st>>>(d, w.xh, w.gu1, w.gf);
  }
  {
    StageScope sc(p, kStGx, st, 2);
    k_gxh<<<dim3((p->N / 2 + 255) / 256, B), 256, 0, st>>>(d, w.gf, gs0, w.gxh);
    k_gx<<<dim3(d.D, B), kFftThreads, (size_t)d.M * 17 / 2, st>>>(d, w.gxh, gs0, gx);
  }
  return cuda_check(cudaGetLastError(), "backward launch");
}

// Time scattering backward: x-hat and U1-hat rebuilt from x and the checkpoint, the second
// order's gY from g_S2t, then the transform's own adjoint chain from gY down to g_x.
jtfs_status launch_scat1d_backward(const jtfs_plan* p, const float* x, const float* u1, int B,
                                   const float* gs0, const float* gs1, const float* gs2t,
                                   float* gx, const Workspace& w, cudaStream_t st) {
  jtfs_status rc = set_attrs(p);
  if (rc != JTFS_OK) return rc;
  const DevPlan& d = p->dp;
  {
    StageScope sc(p, kStXfft, st, 2);
    k_xfft_sub<<<dim3(d.D, B), kFftThreads, (size_t)d.M * 17 / 2, st>>>(d, x, w.xsub);
    k_xfft_combine<<<dim3((p->N / 2 + 255) / 256, B), 256, 0, st>>>(d, w.xsub, w.xh);
  }
  {
    StageScope sc(p, kStUhFromU1, st, 1);
    k_uh_from_u1<<<dim3(p->n1, B), kFftThreads, (size_t)p->L1max * 17 / 2, st>>>(d, u1, w.uh);
  }
  if (gs2t && !p->rowitems.empty()) {
    StageScope sc(p, kStJointBwd, st, 1);
    k_scat1d_bwd_rows<<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                        (size_t)p->rows_cap * 17 / 2, st>>>(
        d, reinterpret_cast<const int4*>(p->d_rowitems), w.uh, gs2t, w.gy);
  } else if (p->y_len > 0) {
    cudaMemsetAsync(w.gy, 0, (size_t)B * p->y_len * sizeof(float2), st);
  }
  {
    StageScope sc(p, kStSecondOrderBwd, st, 2);
    if (!p->rowitems.empty())
      k_gy_spectra<<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                     (size_t)p->rows_cap * 17 / 2, st>>>(
          d, reinterpret_cast<const int4*>(p->d_rowitems), w.gy);
    k_second_order_bwd<<<dim3(p->n1, B), 256, (size_t)p->L1max * 17 / 2, st>>>(d, w.gy, gs1, w.gu1);
  }
  {
    StageScope sc(p, kStStage1Bwd, st, 1);
    k_stage1_bwd<<<dim3(p->n1, B), kRowLaunch, (size_t)p->L1max * 17 / 2, st>>>(d, w.xh, w.gu1, w.gf);
  }
  {
    StageScope sc(p, kStGx, st, 2);
    k_gxh<<<dim3((p->N / 2 + 255) / 256, B), 256, 0, st>>>(d, w.gf, gs0, w.gxh);
    k_gx<<<dim3(d.D, B), kFftThreads, (size_t)d.M * 17 / 2, st>>>(d, w.gxh, gs0, gx);
  }
  return cuda_check(cudaGetLastError(), "time scattering backward");
}

}  // namespace jtfs

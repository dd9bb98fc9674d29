// Kernels shared by the forward and backward passes: the decimated length-N FFT of x,
// the periodisation of x-hat * psi-hat_lambda (Sec. 2) and the second-order time
// wavelet producer Y_alpha (Eq. 3 along t).  Included by both translation units.
#pragma once
#include <cuda_bf16.h>

#include "fft.cuh"
#include "internal.h"

namespace jtfs {
namespace {

constexpr int kFftThreads = 512;
// per-row first-order kernels are launched with 256 threads: with their registers, 512-thread
// blocks leave one block per SM
constexpr int kRowLaunch = 256;

// x-hat by decimation: x_r[m] = x[r + D m] (D sub-sequences of length M), FFT each,
// then x-hat[k] = sum_r exp(-2 pi i r k / N) X_r[k mod M].
__global__ void __launch_bounds__(kFftThreads)
k_xfft_sub(DevPlan P, const float* __restrict__ x, float2* __restrict__ xsub) {
  extern __shared__ float2 sm[];
  const int r = blockIdx.x, b = blockIdx.y;
  const float* xb = x + (size_t)b * P.N;
  for (int m = threadIdx.x; m < P.M; m += blockDim.x)
    sm[fft_pos(bitrev(m, P.logM), P.logM)] = make_float2(__ldg(&xb[r + (size_t)P.D * m]), 0.f);
  __syncthreads();
  fft_dit_rows_r16<-1>(sm, P.logM, 1, twl_for(P, P.logM));
  float2* out = xsub + ((size_t)b * P.D + r) * P.M;
  for (int k = threadIdx.x; k < P.M; k += blockDim.x) out[k] = sm[fft_pos(k, P.logM)];
}

__global__ void k_xfft_combine(DevPlan P, const float2* __restrict__ xsub, float2* __restrict__ xh) {
  const int b = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int half = P.N >> 1;
  if (k >= half) return;
  const int km = k & (P.M - 1);
  const int step = P.TW / P.N;
  const float2* xs = xsub + (size_t)b * P.D * P.M + km;
  float2 acc = make_float2(0.f, 0.f);
  for (int r = 0; r < P.D; ++r) {
    const float2 v = xs[(size_t)r * P.M];
    const int idx = (int)(((long long)r * k) & (P.N - 1)) * step;
    const float2 w = __ldg(&P.tw[idx]);
    acc.x += v.x * w.x - v.y * w.y;
    acc.y += v.x * w.y + v.y * w.x;
  }
  xh[(size_t)b * half + k] = acc;
}

// Periodisation of x-hat * psi-hat_lambda onto L bins: F[k'] = sum_{k = k' mod L} x-hat[k] psi[k],
// written to buf in bit-reversed order (padded layout) for the decimation-in-time inverse FFT.
// Each thread keeps the first terms of eight bins in flight before it sums them (most bins
// take one or two terms); the terms of each bin are added in increasing k.
__device__ __forceinline__ void fold_first_order(const DevPlan& P, const Row1& R,
                                                 const float2* __restrict__ xb, float2* buf) {
  const float* v = P.psi1 + R.off_v;
  const int kend = R.ks + R.kl;
  const int step = blockDim.x;
  for (int base = threadIdx.x; base < R.L; base += 8 * step) {
    float2 a[8];
    float f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kp = base + q * step;
      const int k = R.ks + ((kp - R.ks) & (R.L - 1));
      a[q] = make_float2(0.f, 0.f);
      f[q] = 0.f;
      if (kp < R.L && k < kend) {
        a[q] = xb[k];
        f[q] = __ldg(&v[k - R.ks]);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kp = base + q * step;
      if (kp >= R.L) break;
      float2 acc = make_float2(a[q].x * f[q], a[q].y * f[q]);
      for (int k = R.ks + ((kp - R.ks) & (R.L - 1)) + R.L; k < kend; k += R.L) {
        const float2 t = xb[k];
        const float w = __ldg(&v[k - R.ks]);
        acc.x += t.x * w;
        acc.y += t.y * w;
      }
      buf[fft_pos(bitrev(kp, R.logL), R.logL)] = acc;
    }
  }
}

// Batched Y producer: one CTA takes G consecutive rows lambda'_0 .. lambda'_0 + G - 1 of one
// rate (G L_alpha samples fit the launch's shared memory, padded one per 16), folds them into
// shared memory in bit-reversed order, runs one batched register-radix inverse FFT and writes
// the rows: complex FP32
// (OUT_BF16 = 0), BF16 planes hi (and lo when ylo is given; OUT_BF16 = 1) or FP32 planes
// (OUT_BF16 = 2) in the contraction layout [alpha][2 b + part][lambda' - lam_min][n].  The fold only visits bins below the rate's
// psi-hat support end.
constexpr int kRowThreads = 512;
// launch bound of the row kernels, which run with 256 or 512 threads: declared for 768 so that
// the compiler keeps them within 80 registers, where three 256-thread blocks share an SM (at
// 81 to 96 only two fit)
constexpr int kRowBound = 768;
constexpr int kMaxRowsPerItem = 512;   // G <= rows_cap / 32

// Folds the G rows lam0 .. lam0 + G - 1 of rate a (U1-hat * psi-hat_alpha onto L_alpha bins)
// into sm in bit-reversed padded order and runs their batched inverse FFT; s_inv[r] receives
// the scale 1 / L of first-order row lam0 + r.  The producer of Y_alpha and the time-scattering
// kernels share it.
__device__ __forceinline__ void second_order_rows_ifft(const DevPlan& P, const Rate2& A, int a,
                                                       int lam0, int G, const float2* ub,
                                                       float2* sm, int* s_off, int* s_kend,
                                                       float* s_inv) {
  const float* psi = P.psi2 + (size_t)a * P.K2max;
  const int L = A.L, logL = A.logL;
  for (int r = threadIdx.x; r < G; r += blockDim.x) {
    const Row1 R = P.rows1[lam0 + r];
    s_off[r] = R.off_uh;
    s_kend[r] = min(R.L >> 1, A.k2e);
    s_inv[r] = 1.f / (float)R.L;
  }
  __syncthreads();
  // the first terms of eight bins per thread in flight before they are summed (a bin takes
  // one term below the filter's support end, further ones only where that end passes L)
  const int total = G * L, step = blockDim.x;
  for (int base = threadIdx.x; base < total; base += 8 * step) {
    float2 u[8];
    float f[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = base + q * step;
      u[q] = make_float2(0.f, 0.f);
      f[q] = 0.f;
      if (idx < total) {
        const int row = idx >> logL, kp = idx & (L - 1);
        if (kp < s_kend[row]) {
          u[q] = ub[s_off[row] + kp];
          f[q] = __ldg(&psi[kp]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = base + q * step;
      if (idx >= total) break;
      const int row = idx >> logL, kp = idx & (L - 1);
      const float2* ur = ub + s_off[row];
      const int kend = s_kend[row];
      float2 acc = make_float2(u[q].x * f[q], u[q].y * f[q]);
      for (int k = kp + L; k < kend; k += L) {
        const float2 t = ur[k];
        const float w = __ldg(&psi[k]);
        acc.x += t.x * w;
        acc.y += t.y * w;
      }
      sm[fft_pos((row << logL) + bitrev(kp, logL), logL)] = acc;
    }
  }
  __syncthreads();
  fft_dit_rows_r16<+1>(sm, logL, G, twl_for(P, logL));
}

template <int OUT_BF16>
__global__ void __launch_bounds__(kRowBound)
k_second_order_rows(DevPlan P, const int4* __restrict__ items, const float2* __restrict__ uh,
                    float2* __restrict__ y, __nv_bfloat16* __restrict__ yhi,
                    __nv_bfloat16* __restrict__ ylo, int B) {
  extern __shared__ float2 sm[];
  __shared__ int s_off[kMaxRowsPerItem], s_kend[kMaxRowsPerItem];
  __shared__ float s_inv[kMaxRowsPerItem];
  const int4 it = items[blockIdx.x];
  const int a = it.x, lam0 = it.y, G = it.z, b = blockIdx.y;
  const Rate2 A = P.rates2[a];
  const int L = A.L, logL = A.logL;
  second_order_rows_ifft(P, A, a, lam0, G, uh + (size_t)b * P.uh_len, sm, s_off, s_kend, s_inv);
  if (OUT_BF16 == 0) {
    float2* ya = y + (size_t)b * P.y_len + A.off_y + (size_t)(lam0 - A.lam_min) * L;
    for (int idx = threadIdx.x; idx < G * L; idx += blockDim.x) {
      const float inv = s_inv[idx >> logL];
      const float2 v = sm[fft_pos(idx, logL)];
      ya[idx] = make_float2(v.x * inv, v.y * inv);
    }
  } else if (OUT_BF16 == 2) {
    // FP32 planes in the contraction layout (the TF32 operands)
    float* yf = reinterpret_cast<float*>(y);
    const size_t plane = (size_t)A.K * L;
    const size_t base = (size_t)B * 2 * A.off_y + (size_t)(2 * b) * plane + (size_t)(lam0 - A.lam_min) * L;
    for (int i2 = threadIdx.x; i2 < (G * L) >> 1; i2 += blockDim.x) {
      const int idx = 2 * i2;
      const float inv = s_inv[idx >> logL];
      const float2 v0 = sm[fft_pos(idx, logL)], v1 = sm[fft_pos(idx + 1, logL)];
      *reinterpret_cast<float2*>(yf + base + idx) = make_float2(v0.x * inv, v1.x * inv);
      *reinterpret_cast<float2*>(yf + base + plane + idx) = make_float2(v0.y * inv, v1.y * inv);
    }
  } else {
    // rows of one rate are contiguous in each plane: element idx of the block sits at
    // (lam0 - lam_min) L + idx
    const size_t plane = (size_t)A.K * L;
    const size_t base = (size_t)B * 2 * A.off_y + (size_t)(2 * b) * plane + (size_t)(lam0 - A.lam_min) * L;
    // four samples per thread, one 8-byte store per plane, where rows hold at least four
    // samples (so a group never straddles rows) and both plane offsets are multiples of four
    // samples; else two samples per thread
    const bool quad = L >= 4 && (base & 3) == 0 && (plane & 3) == 0;
    for (int i2 = threadIdx.x; !quad && i2 < (G * L) >> 1; i2 += blockDim.x) {
      const int idx = 2 * i2;
      const float inv = s_inv[idx >> logL];
      const float2 v0 = sm[fft_pos(idx, logL)], v1 = sm[fft_pos(idx + 1, logL)];
      const float r0 = v0.x * inv, r1 = v1.x * inv, i0 = v0.y * inv, i1 = v1.y * inv;
      const __nv_bfloat162 hr = __floats2bfloat162_rn(r0, r1), hi_ = __floats2bfloat162_rn(i0, i1);
      *reinterpret_cast<__nv_bfloat162*>(yhi + base + idx) = hr;
      *reinterpret_cast<__nv_bfloat162*>(yhi + base + plane + idx) = hi_;
      if (ylo) {
        const float2 fr = __bfloat1622float2(hr), fi = __bfloat1622float2(hi_);
        *reinterpret_cast<__nv_bfloat162*>(ylo + base + idx) = __floats2bfloat162_rn(r0 - fr.x, r1 - fr.y);
        *reinterpret_cast<__nv_bfloat162*>(ylo + base + plane + idx) = __floats2bfloat162_rn(i0 - fi.x, i1 - fi.y);
      }
    }
    for (int i4 = threadIdx.x; quad && i4 < (G * L) >> 2; i4 += blockDim.x) {
      const int idx = 4 * i4;
      const float inv = s_inv[idx >> logL];
      uint32_t hw[2][2], lw[2][2];   // [re / im][sample pair]
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const float2 v0 = sm[fft_pos(idx + 2 * e, logL)], v1 = sm[fft_pos(idx + 2 * e + 1, logL)];
        const float r0 = v0.x * inv, r1 = v1.x * inv, i0 = v0.y * inv, i1 = v1.y * inv;
        const __nv_bfloat162 hr = __floats2bfloat162_rn(r0, r1), hi_ = __floats2bfloat162_rn(i0, i1);
        hw[0][e] = *reinterpret_cast<const uint32_t*>(&hr);
        hw[1][e] = *reinterpret_cast<const uint32_t*>(&hi_);
        const float2 fr = __bfloat1622float2(hr), fi = __bfloat1622float2(hi_);
        const __nv_bfloat162 lr = __floats2bfloat162_rn(r0 - fr.x, r1 - fr.y);
        const __nv_bfloat162 li = __floats2bfloat162_rn(i0 - fi.x, i1 - fi.y);
        lw[0][e] = *reinterpret_cast<const uint32_t*>(&lr);
        lw[1][e] = *reinterpret_cast<const uint32_t*>(&li);
      }
      *reinterpret_cast<uint2*>(yhi + base + idx) = make_uint2(hw[0][0], hw[0][1]);
      *reinterpret_cast<uint2*>(yhi + base + plane + idx) = make_uint2(hw[1][0], hw[1][1]);
      if (ylo) {
        *reinterpret_cast<uint2*>(ylo + base + idx) = make_uint2(lw[0][0], lw[0][1]);
        *reinterpret_cast<uint2*>(ylo + base + plane + idx) = make_uint2(lw[1][0], lw[1][1]);
      }
    }
  }
}

}  // namespace
}  // namespace jtfs

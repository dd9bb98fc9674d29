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

// x-hat by decimation: x_r[m] = x[r + D m] (D sub-sequences of length M), FFT each,
// then x-hat[k] = sum_r exp(-2 pi i r k / N) X_r[k mod M].
__global__ void __launch_bounds__(kFftThreads)
k_xfft_sub(DevPlan P, const float* __restrict__ x, float2* __restrict__ xsub) {
  extern __shared__ float2 sm[];
  const int r = blockIdx.x, b = blockIdx.y;
  const float* xb = x + (size_t)b * P.N;
  for (int m = threadIdx.x; m < P.M; m += blockDim.x)
    sm[m] = make_float2(__ldg(&xb[r + (size_t)P.D * m]), 0.f);
  __syncthreads();
  fft_dif<-1>(sm, P.logM, P.tw, P.logTW);
  float2* out = xsub + ((size_t)b * P.D + r) * P.M;
  for (int k = threadIdx.x; k < P.M; k += blockDim.x) out[k] = sm[bitrev(k, P.logM)];
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
// written to buf in bit-reversed order for the decimation-in-time inverse FFT.
__device__ __forceinline__ void fold_first_order(const DevPlan& P, const Row1& R,
                                                 const float2* __restrict__ xb, float2* buf) {
  const float* v = P.psi1 + R.off_v;
  const int kend = R.ks + R.kl;
  for (int kp = threadIdx.x; kp < R.L; kp += blockDim.x) {
    int k = R.ks + ((kp - R.ks) & (R.L - 1));
    float2 acc = make_float2(0.f, 0.f);
    for (; k < kend; k += R.L) {
      const float2 a = xb[k];
      const float f = __ldg(&v[k - R.ks]);
      acc.x += a.x * f;
      acc.y += a.y * f;
    }
    buf[bitrev(kp, R.logL)] = acc;
  }
}

// Y_alpha row of lambda': the row spectrum U1-hat[k] (positive bins below the row's Nyquist)
// times psi-hat_alpha(k / N), folded modulo L_alpha, inverse FFT, scaled by 1 / L_lambda'.
// OUT_BF16 = 0: Y row written as complex FP32 at the per-signal offset of the rate.
// OUT_BF16 = 1: Y row written as BF16 planes for the tensor-core contraction, layout
// [alpha][2 b + part][lambda' - lam_min][n] (part 0 = Re, 1 = Im), value = hi + lo with
// hi = bf16(v) and lo = bf16(v - hi).
template <int OUT_BF16>
__global__ void __launch_bounds__(kFftThreads)
k_second_order(DevPlan P, const int2* __restrict__ pairs, const float2* __restrict__ uh,
               float2* __restrict__ y, __nv_bfloat16* __restrict__ yhi,
               __nv_bfloat16* __restrict__ ylo, int B) {
  extern __shared__ float2 sm[];
  const int2 pr = pairs[blockIdx.x];
  const int a = pr.x, lam = pr.y, b = blockIdx.y;
  const Row1 R = P.rows1[lam];
  const Rate2 A = P.rates2[a];
  const float2* ur = uh + (size_t)b * P.uh_len + R.off_uh;
  const float* psi = P.psi2 + (size_t)a * P.K2max;
  const int kmax = R.L >> 1;  // positive frequencies strictly below the row's Nyquist
  for (int kp = threadIdx.x; kp < A.L; kp += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int k = kp; k < kmax; k += A.L) {
      const float2 u = ur[k];
      const float f = __ldg(&psi[k]);
      acc.x += u.x * f;
      acc.y += u.y * f;
    }
    sm[bitrev(kp, A.logL)] = acc;
  }
  __syncthreads();
  fft_dit<+1>(sm, A.logL, P.tw, P.logTW);
  const float inv = 1.f / (float)R.L;
  if (!OUT_BF16) {
    float2* yr = y + (size_t)b * P.y_len + A.off_y + (size_t)(lam - A.lam_min) * A.L;
    for (int m = threadIdx.x; m < A.L; m += blockDim.x) {
      const float2 v = sm[m];
      yr[m] = make_float2(v.x * inv, v.y * inv);
    }
  } else {
    const size_t region = (size_t)B * 2 * A.off_y;
    const size_t plane = (size_t)A.K * A.L;
    const size_t off_re = region + (size_t)(2 * b) * plane + (size_t)(lam - A.lam_min) * A.L;
    const size_t off_im = off_re + plane;
    for (int m = threadIdx.x; m < A.L; m += blockDim.x) {
      const float2 v = sm[m];
      const float re = v.x * inv, im = v.y * inv;
      const __nv_bfloat16 hr = __float2bfloat16_rn(re), hi_ = __float2bfloat16_rn(im);
      yhi[off_re + m] = hr;
      yhi[off_im + m] = hi_;
      if (ylo) {
        ylo[off_re + m] = __float2bfloat16_rn(re - __bfloat162float(hr));
        ylo[off_im + m] = __float2bfloat16_rn(im - __bfloat162float(hi_));
      }
    }
  }
}

// Batched Y producer: one CTA takes G consecutive rows lambda'_0 .. lambda'_0 + G - 1 of one rate
// (G L_alpha <= 8192 samples), folds them into shared memory, runs one batched inverse FFT and
// writes BF16 planes (hi, and lo when ylo is given) or complex FP32 rows.
constexpr int kRowThreads = 256;

template <int OUT_BF16>
__global__ void __launch_bounds__(kRowThreads)
k_second_order_rows(DevPlan P, const int4* __restrict__ items, const float2* __restrict__ uh,
                    float2* __restrict__ y, __nv_bfloat16* __restrict__ yhi,
                    __nv_bfloat16* __restrict__ ylo, int B) {
  extern __shared__ float2 sm[];
  const int4 it = items[blockIdx.x];
  const int a = it.x, lam0 = it.y, G = it.z, b = blockIdx.y;
  const Rate2 A = P.rates2[a];
  const float* psi = P.psi2 + (size_t)a * P.K2max;
  const int L = A.L, logL = A.logL;
  for (int idx = threadIdx.x; idx < G * L; idx += blockDim.x) {
    const int row = idx >> logL, kp = idx & (L - 1);
    const Row1 R = P.rows1[lam0 + row];
    const float2* ur = uh + (size_t)b * P.uh_len + R.off_uh;
    const int kmax = R.L >> 1;
    float2 acc = make_float2(0.f, 0.f);
    for (int k = kp; k < kmax; k += L) {
      const float2 u = ur[k];
      const float f = __ldg(&psi[k]);
      acc.x += u.x * f;
      acc.y += u.y * f;
    }
    sm[(row << logL) + bitrev(kp, logL)] = acc;
  }
  __syncthreads();
  fft_dit_rows<+1>(sm, logL, G, P.tw, P.logTW);
  if (!OUT_BF16) {
    for (int idx = threadIdx.x; idx < G * L; idx += blockDim.x) {
      const int row = idx >> logL, m = idx & (L - 1);
      const float inv = 1.f / (float)P.rows1[lam0 + row].L;
      const float2 v = sm[idx];
      y[(size_t)b * P.y_len + A.off_y + (size_t)(lam0 + row - A.lam_min) * L + m] =
          make_float2(v.x * inv, v.y * inv);
    }
  } else {
    const size_t region = (size_t)B * 2 * A.off_y;
    const size_t plane = (size_t)A.K * L;
    for (int idx = threadIdx.x; idx < G * L; idx += blockDim.x) {
      const int row = idx >> logL, m = idx & (L - 1);
      const float inv = 1.f / (float)P.rows1[lam0 + row].L;
      const size_t off_re = region + (size_t)(2 * b) * plane + (size_t)(lam0 + row - A.lam_min) * L + m;
      const size_t off_im = off_re + plane;
      const float2 v = sm[idx];
      const float re = v.x * inv, im = v.y * inv;
      const __nv_bfloat16 hr = __float2bfloat16_rn(re), hi_ = __float2bfloat16_rn(im);
      yhi[off_re] = hr;
      yhi[off_im] = hi_;
      if (ylo) {
        ylo[off_re] = __float2bfloat16_rn(re - __bfloat162float(hr));
        ylo[off_im] = __float2bfloat16_rn(im - __bfloat162float(hi_));
      }
    }
  }
}

}  // namespace
}  // namespace jtfs

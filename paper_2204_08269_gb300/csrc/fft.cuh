// Shared-memory complex FFTs of power-of-two length, written from the Cooley-Tukey
// factorisation.  Twiddles come from a table tw[j] = exp(-2 pi i j / TW) built in FP64 on
// the host; a stage of span 2^s reads tw[j * TW / 2^s].
//
// fft_dit: input in bit-reversed order, output in natural order (decimation in time).
// fft_dif: input in natural order, output in bit-reversed order (decimation in frequency).
// SIGN = -1 computes sum_n v[n] exp(-2 pi i k n / L); SIGN = +1 the conjugate kernel (no 1/L).
// Both must be called by every thread of the block; they end with __syncthreads().
#pragma once
#include <cuda_runtime.h>

namespace jtfs {

__device__ __forceinline__ int bitrev(int k, int logL) {
  return logL ? (int)(__brev((unsigned)k) >> (32 - logL)) : 0;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

template <int SIGN>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int idx) {
  float2 w = __ldg(&tw[idx]);
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// Radix-4 butterflies where possible (two radix-2 stages fused), radix-2 for an odd stage.
template <int SIGN>
__device__ void fft_dit(float2* buf, int logL, const float2* __restrict__ tw, int logTW) {
  const int L = 1 << logL;
  int s = 1;
  if (logL & 1) {  // one radix-2 stage of span 2 (twiddle 1)
    for (int b = threadIdx.x; b < (L >> 1); b += blockDim.x) {
      const int i0 = b << 1;
      const float2 a = buf[i0], c = buf[i0 + 1];
      buf[i0] = make_float2(a.x + c.x, a.y + c.y);
      buf[i0 + 1] = make_float2(a.x - c.x, a.y - c.y);
    }
    __syncthreads();
    s = 2;
  }
  // fused stages (s, s+1): span 2^(s+1), quarter q = 2^(s-1)
  for (; s + 1 <= logL; s += 2) {
    const int q = 1 << (s - 1);
    const int sh1 = logTW - s;        // twiddle of stage s:   tw[j << sh1], j < q
    const int sh2 = logTW - s - 1;    // twiddle of stage s+1: tw[j << sh2], j < 2q
    for (int b = threadIdx.x; b < (L >> 2); b += blockDim.x) {
      const int j = b & (q - 1);
      const int base = ((b >> (s - 1)) << (s + 1)) | j;
      float2 x0 = buf[base], x1 = buf[base + q], x2 = buf[base + 2 * q], x3 = buf[base + 3 * q];
      // stage s on pairs (x0,x1) and (x2,x3), twiddle w1 = W_{2q}^j
      const float2 w1 = twiddle<SIGN>(tw, j << sh1);
      float2 t = cmul(x1, w1);
      float2 a0 = make_float2(x0.x + t.x, x0.y + t.y), a1 = make_float2(x0.x - t.x, x0.y - t.y);
      t = cmul(x3, w1);
      float2 a2 = make_float2(x2.x + t.x, x2.y + t.y), a3 = make_float2(x2.x - t.x, x2.y - t.y);
      // stage s+1 on pairs (a0,a2) with W_{4q}^j and (a1,a3) with W_{4q}^{j+q}
      const float2 w2 = twiddle<SIGN>(tw, j << sh2);
      const float2 w3 = twiddle<SIGN>(tw, (j + q) << sh2);
      t = cmul(a2, w2);
      buf[base] = make_float2(a0.x + t.x, a0.y + t.y);
      buf[base + 2 * q] = make_float2(a0.x - t.x, a0.y - t.y);
      t = cmul(a3, w3);
      buf[base + q] = make_float2(a1.x + t.x, a1.y + t.y);
      buf[base + 3 * q] = make_float2(a1.x - t.x, a1.y - t.y);
    }
    __syncthreads();
  }
}

template <int SIGN>
__device__ void fft_dif(float2* buf, int logL, const float2* __restrict__ tw, int logTW) {
  const int L = 1 << logL;
  int s = logL;
  // fused stages (s, s-1): span 2^s, quarter q = 2^(s-2)
  for (; s - 1 >= 1; s -= 2) {
    const int q = 1 << (s - 2);
    const int sh1 = logTW - s;        // stage s twiddles tw[j << sh1], j < 2q
    const int sh2 = logTW - s + 1;    // stage s-1 twiddles tw[j << sh2], j < q
    for (int b = threadIdx.x; b < (L >> 2); b += blockDim.x) {
      const int j = b & (q - 1);
      const int base = ((b >> (s - 2)) << s) | j;
      float2 x0 = buf[base], x1 = buf[base + q], x2 = buf[base + 2 * q], x3 = buf[base + 3 * q];
      // stage s: pairs (x0,x2) with W_{4q}^j, (x1,x3) with W_{4q}^{j+q}
      const float2 w1 = twiddle<SIGN>(tw, j << sh1);
      const float2 w1b = twiddle<SIGN>(tw, (j + q) << sh1);
      float2 a0 = make_float2(x0.x + x2.x, x0.y + x2.y);
      float2 a2 = cmul(make_float2(x0.x - x2.x, x0.y - x2.y), w1);
      float2 a1 = make_float2(x1.x + x3.x, x1.y + x3.y);
      float2 a3 = cmul(make_float2(x1.x - x3.x, x1.y - x3.y), w1b);
      // stage s-1: pairs (a0,a1) and (a2,a3) with W_{2q}^j
      const float2 w2 = twiddle<SIGN>(tw, j << sh2);
      buf[base] = make_float2(a0.x + a1.x, a0.y + a1.y);
      buf[base + q] = cmul(make_float2(a0.x - a1.x, a0.y - a1.y), w2);
      buf[base + 2 * q] = make_float2(a2.x + a3.x, a2.y + a3.y);
      buf[base + 3 * q] = cmul(make_float2(a2.x - a3.x, a2.y - a3.y), w2);
    }
    __syncthreads();
  }
  if (s == 1) {  // last radix-2 stage of span 2 (twiddle 1)
    for (int b = threadIdx.x; b < (L >> 1); b += blockDim.x) {
      const int i0 = b << 1;
      const float2 a = buf[i0], c = buf[i0 + 1];
      buf[i0] = make_float2(a.x + c.x, a.y + c.y);
      buf[i0 + 1] = make_float2(a.x - c.x, a.y - c.y);
    }
    __syncthreads();
  }
}

}  // namespace jtfs

namespace jtfs {

// Batched forms: G independent rows of length L = 2^logL stored back to back in buf, every
// thread of the block working on butterflies of all rows.  Same decimation as above.
template <int SIGN>
__device__ void fft_dit_rows(float2* buf, int logL, int G, const float2* __restrict__ tw,
                             int logTW) {
  const int L = 1 << logL;
  int s = 1;
  if (logL & 1) {
    const int per = L >> 1;
    for (int b = threadIdx.x; b < G * per; b += blockDim.x) {
      const int i0 = ((b >> (logL - 1)) << logL) + ((b & (per - 1)) << 1);
      const float2 a = buf[i0], c = buf[i0 + 1];
      buf[i0] = make_float2(a.x + c.x, a.y + c.y);
      buf[i0 + 1] = make_float2(a.x - c.x, a.y - c.y);
    }
    __syncthreads();
    s = 2;
  }
  const int per = L >> 2;
  for (; s + 1 <= logL; s += 2) {
    const int q = 1 << (s - 1);
    const int sh1 = logTW - s;
    const int sh2 = logTW - s - 1;
    for (int bb = threadIdx.x; bb < G * per; bb += blockDim.x) {
      const int row = bb >> (logL - 2), b = bb & (per - 1);
      const int j = b & (q - 1);
      const int base = (row << logL) + (((b >> (s - 1)) << (s + 1)) | j);
      float2 x0 = buf[base], x1 = buf[base + q], x2 = buf[base + 2 * q], x3 = buf[base + 3 * q];
      const float2 w1 = twiddle<SIGN>(tw, j << sh1);
      float2 t = cmul(x1, w1);
      float2 a0 = make_float2(x0.x + t.x, x0.y + t.y), a1 = make_float2(x0.x - t.x, x0.y - t.y);
      t = cmul(x3, w1);
      float2 a2 = make_float2(x2.x + t.x, x2.y + t.y), a3 = make_float2(x2.x - t.x, x2.y - t.y);
      const float2 w2 = twiddle<SIGN>(tw, j << sh2);
      const float2 w3 = twiddle<SIGN>(tw, (j + q) << sh2);
      t = cmul(a2, w2);
      buf[base] = make_float2(a0.x + t.x, a0.y + t.y);
      buf[base + 2 * q] = make_float2(a0.x - t.x, a0.y - t.y);
      t = cmul(a3, w3);
      buf[base + q] = make_float2(a1.x + t.x, a1.y + t.y);
      buf[base + 3 * q] = make_float2(a1.x - t.x, a1.y - t.y);
    }
    __syncthreads();
  }
}

template <int SIGN>
__device__ void fft_dif_rows(float2* buf, int logL, int G, const float2* __restrict__ tw,
                             int logTW) {
  const int L = 1 << logL;
  int s = logL;
  const int per = L >> 2;
  for (; s - 1 >= 1; s -= 2) {
    const int q = 1 << (s - 2);
    const int sh1 = logTW - s;
    const int sh2 = logTW - s + 1;
    for (int bb = threadIdx.x; bb < G * per; bb += blockDim.x) {
      const int row = bb >> (logL - 2), b = bb & (per - 1);
      const int j = b & (q - 1);
      const int base = (row << logL) + (((b >> (s - 2)) << s) | j);
      float2 x0 = buf[base], x1 = buf[base + q], x2 = buf[base + 2 * q], x3 = buf[base + 3 * q];
      const float2 w1 = twiddle<SIGN>(tw, j << sh1);
      const float2 w1b = twiddle<SIGN>(tw, (j + q) << sh1);
      float2 a0 = make_float2(x0.x + x2.x, x0.y + x2.y);
      float2 a2 = cmul(make_float2(x0.x - x2.x, x0.y - x2.y), w1);
      float2 a1 = make_float2(x1.x + x3.x, x1.y + x3.y);
      float2 a3 = cmul(make_float2(x1.x - x3.x, x1.y - x3.y), w1b);
      const float2 w2 = twiddle<SIGN>(tw, j << sh2);
      buf[base] = make_float2(a0.x + a1.x, a0.y + a1.y);
      buf[base + q] = cmul(make_float2(a0.x - a1.x, a0.y - a1.y), w2);
      buf[base + 2 * q] = make_float2(a2.x + a3.x, a2.y + a3.y);
      buf[base + 3 * q] = cmul(make_float2(a2.x - a3.x, a2.y - a3.y), w2);
    }
    __syncthreads();
  }
  if (s == 1) {
    const int per2 = L >> 1;
    for (int b = threadIdx.x; b < G * per2; b += blockDim.x) {
      const int i0 = ((b >> (logL - 1)) << logL) + ((b & (per2 - 1)) << 1);
      const float2 a = buf[i0], c = buf[i0 + 1];
      buf[i0] = make_float2(a.x + c.x, a.y + c.y);
      buf[i0 + 1] = make_float2(a.x - c.x, a.y - c.y);
    }
    __syncthreads();
  }
}

}  // namespace jtfs

namespace jtfs {

// Register-radix forms for a padded layout: element i of a row block lives at
// fft_pad(i) = i + i / 16 (one float2 of padding per 16), which keeps the strided accesses
// of the first passes free of bank conflicts.  A pass fuses RB consecutive radix-2 DIT
// stages s0 .. s0 + RB - 1 in registers: each thread loads 2^RB elements at stride
// q = 2^(s0-1), applies the stages with the twiddles of the L-point table tw
// (exp(-2 pi i m / L), m < L / 2) and stores them back.
__device__ __forceinline__ int fft_pad(int i) { return i + (i >> 4); }

template <int SIGN, int RB>
__device__ __forceinline__ void fft_dit_pass(float2* buf, int logL, int G,
                                             const float2* __restrict__ tw, int s0) {
  constexpr int R = 1 << RB;
  const int q = 1 << (s0 - 1);
  const int lgpr = logL - RB;                 // log2 of the groups per row
  const int groups = G << lgpr;
  for (int g = threadIdx.x; g < groups; g += blockDim.x) {
    const int row = g >> lgpr, b = g & ((1 << lgpr) - 1);
    const int j = b & (q - 1);
    const int base = (row << logL) + ((b >> (s0 - 1)) << (s0 - 1 + RB)) + j;
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = buf[fft_pad(base + m * q)];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int sh = logL - s0 - u;
      float2 w[1 << (RB - 1)];
#pragma unroll
      for (int ml = 0; ml < (1 << u); ++ml) w[ml] = twiddle<SIGN>(tw, (j + q * ml) << sh);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (m & (1 << u)) continue;
        const int mp = m + (1 << u);
        const float2 t = cmul(v[mp], w[m & ((1 << u) - 1)]);
        v[mp] = make_float2(v[m].x - t.x, v[m].y - t.y);
        v[m] = make_float2(v[m].x + t.x, v[m].y + t.y);
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) buf[fft_pad(base + m * q)] = v[m];
  }
  __syncthreads();
}

// G rows of length 2^logL (padded layout, bit-reversed input, natural output): a first pass
// of logL mod 4 stages, then radix-16 passes.  Every thread of the block must call it.
template <int SIGN>
__device__ void fft_dit_rows_r16(float2* buf, int logL, int G, const float2* __restrict__ tw) {
  int s0 = 1;
  switch (logL & 3) {
    case 1: fft_dit_pass<SIGN, 1>(buf, logL, G, tw, s0); s0 += 1; break;
    case 2: fft_dit_pass<SIGN, 2>(buf, logL, G, tw, s0); s0 += 2; break;
    case 3: fft_dit_pass<SIGN, 3>(buf, logL, G, tw, s0); s0 += 3; break;
    default: break;
  }
  for (; s0 + 3 <= logL; s0 += 4) fft_dit_pass<SIGN, 4>(buf, logL, G, tw, s0);
}

}  // namespace jtfs

// Shared-memory complex FFTs of power-of-two length, written from the Cooley-Tukey
// factorisation (decimation in time: bit-reversed input, natural-order output).  Twiddles
// come from the per-length table tw[m] = exp(-2 pi i m / L), m < L / 2, built in FP64 on
// the host; a stage of span 2^s reads tw[j * L / 2^s].
// SIGN = -1 computes sum_n v[n] exp(-2 pi i k n / L); SIGN = +1 the conjugate kernel (no 1/L).
// Every thread of the block must call them; they end with __syncthreads().
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

// Complex sums as packed FP32 pairs (one instruction each, sm_100 and later); a - b is taken
// as b * (-1) + a, whose product is exact, so it rounds like a - b.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

template <int SIGN>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int idx) {
  float2 w = __ldg(&tw[idx]);
  if (SIGN > 0) w.y = -w.y;
  return w;
}

}  // namespace jtfs

namespace jtfs {

// Register-radix forms for a padded layout: element i of a row block lives at fft_pos(i, logL)
// (below: one float2 of padding per 16, plus an XOR of index bits for long rows), which keeps
// the strided accesses of the passes free of bank conflicts.  A pass fuses RB consecutive radix-2 DIT
// stages s0 .. s0 + RB - 1 in registers: each thread loads 2^RB elements at stride
// q = 2^(s0-1), applies the stages with the twiddles of the L-point table tw
// (exp(-2 pi i m / L), m < L / 2; one entry per stage, the others by fixed unit roots) and
// stores them back.
__device__ __forceinline__ int fft_pad(int i) { return i + (i >> 4); }

// Shared-memory position of element i of a block of rows of 2^logL elements: fft_pad, and for
// rows of 512 or more the top four bits of i's index within its row XORed into its low four
// bits first.  The bit-reversed scatters of the inputs send a half-warp's 16 consecutive bins
// to indices that differ only in their top bits, which fft_pad alone maps to one bank (2- to
// 16-way conflicts for rows of 1024 to 16384); the XOR spreads them over all banks, and the
// strided accesses of the passes and the natural-order reads stay conflict-free (a model of
// the 8-byte bank mapping over logL = 5 .. 15; at logL = 8 the XOR would conflict instead).
// Within a row it is a bijection onto the same positions as fft_pad.
__device__ __forceinline__ int fft_pos(int i, int logL) {
  if (logL >= 9) i ^= (i >> (logL - 4)) & 15;
  return i + (i >> 4);
}

// exp(-i pi m / 2^u) for u = 1..3 and 0 < m < 2^u (conjugated for SIGN = +1): within a
// pass, the twiddles of stage u are the table entry of the group times these roots.
template <int SIGN>
__device__ __forceinline__ float2 unit_root(int u, int m) {
  constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f;   // cos, sin(pi/8)
  constexpr float h = 0.70710678118654752f;                               // cos(pi/4)
  float2 r = make_float2(1.f, 0.f);
  const int e = m << (3 - u);                 // angle -pi e / 8, e = 1..7
  switch (e) {
    case 1: r = make_float2(c1, -s1); break;
    case 2: r = make_float2(h, -h); break;
    case 3: r = make_float2(s1, -c1); break;
    case 4: r = make_float2(0.f, -1.f); break;
    case 5: r = make_float2(-s1, -c1); break;
    case 6: r = make_float2(-h, -h); break;
    case 7: r = make_float2(-c1, -s1); break;
    default: break;
  }
  if (SIGN > 0) r.y = -r.y;
  return r;
}

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
    // p[m] = fft_pos(base + m q, logL), from fewer operations: below the last pass of a
    // swizzled row the XOR term t (the top four in-row bits) is the same for the whole group,
    // and from q = 16 on the positions step by q + q / 16; in the last radix-16 pass of a
    // swizzled row (base = j < q) the term is m itself
    int p[R];
    if (logL >= 9 && RB == 4 && s0 + 3 == logL) {
      const int c0 = (row << logL) + (row << (logL - 4)) + (j >> 4);
#pragma unroll
      for (int m = 0; m < R; ++m) p[m] = c0 + (j ^ m) + m * (q + (q >> 4));
    } else if (logL < 9 || s0 + RB - 1 <= logL - 4) {
      const int t = logL >= 9 ? (base >> (logL - 4)) & 15 : 0;
      if (q >= 16) {
        const int p0 = fft_pad(base ^ t);
#pragma unroll
        for (int m = 0; m < R; ++m) p[m] = p0 + m * (q + (q >> 4));
      } else {
#pragma unroll
        for (int m = 0; m < R; ++m) p[m] = fft_pad((base + m * q) ^ t);
      }
    } else {
#pragma unroll
      for (int m = 0; m < R; ++m) p[m] = fft_pos(base + m * q, logL);
    }
    float2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = buf[p[m]];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int sh = logL - s0 - u;
      // w[ml] = tw[(j + q ml) << sh] = tw[j << sh] exp(-i pi ml / 2^u)
      float2 w[1 << (RB - 1)];
      w[0] = twiddle<SIGN>(tw, j << sh);
#pragma unroll
      for (int ml = 1; ml < (1 << u); ++ml) w[ml] = cmul(w[0], unit_root<SIGN>(u, ml));
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if (m & (1 << u)) continue;
        const int mp = m + (1 << u);
        const float2 t = cmul(v[mp], w[m & ((1 << u) - 1)]);
        v[mp] = csub(v[m], t);
        v[m] = cadd(v[m], t);
      }
    }
#pragma unroll
    for (int m = 0; m < R; ++m) buf[p[m]] = v[m];
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

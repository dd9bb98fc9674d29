// Tensor-core (tcgen05) forward of the joint stage (Eq. 2-3): for every rate alpha, signal b
// and tile of 128 stacked channel rows r = c * n1 + lambda,
//     Z[r, n] = sum_lambda' W[r, lambda'] Y_alpha[lambda', n]      (complex, K = lambda')
// with W[c * n1 + lambda, lambda'] = h_c[(lambda - lambda') mod N_fr], then |Z| and the phi_T
// Riemann sum over n, accumulated per row across every column tile of the signal:
//     P[b, alpha, r, t] = sum_n w_alpha[n, t] |Z[r, n]|.
// A separate small kernel applies the phi_F pooling along lambda (or none, Eq. 4).
//
// Operands are BF16 planes (Re / Im, and a low-order plane each for the three-pass split
// x = hi + lo that gives FP32-level accuracy: hi*hi + hi*lo + lo*hi).  W planes are K-major
// (lambda' contiguous, 64-byte swizzle, 32 lambda' per stage); Y planes are MN-major (time
// contiguous, 128-byte swizzle), exactly the layout the second-order producer writes.
// Complex product from real MMAs into two TMEM accumulators, using the descriptor's
// negate-A bit:  Re += Wr Yr + (-Wi) Yi,  Im += Wr Yi + Wi Yr.
//
// Column tiles are BN = 128 samples wide when the pooled frame count is 16 (the MMAs then
// run at the full tensor rate; an M = 128, K = 16 MMA costs the same ~47 cycles for any
// N <= 64) and 64 wide otherwise.  One accumulator (Re, Im: 2 BN TMEM columns) is released as
// soon as the epilogue has loaded it, so the next tile's product overlaps the modulus.
//
// Roles (576 threads): warp 0 = TMA producer, warp 1 = MMA issuer (and TMEM owner),
// warps 2..17 = epilogue (four warps per TMEM lane quarter, BN / 4 columns each).
// Every wait is bounded; on timeout the CTA records an error code and unwinds.
#include <cuda_bf16.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fft.cuh"
#include "internal.h"
#include "tma_host.h"
#include "umma.cuh"

namespace jtfs {

using namespace umma;

namespace {

constexpr int kBM = 128, kBK = 32;
constexpr int kEpiWarp0 = 2, kEpiWarps = 16;
constexpr int kThreads = 32 * (kEpiWarp0 + kEpiWarps);
constexpr int kMaxWS = 4;                     // pooling-weight ring depth (at most)

struct TcMaps {
  CUtensorMap w[4];        // Wr_hi, Wi_hi, Wr_lo, Wi_lo : [C*n1 rows][n1_pad] bf16, box {32, 128}
  CUtensorMap y[2][16];    // [hi/lo][alpha] : [2B][K_alpha][L_alpha] bf16, box {64, 32, 1}
  CUtensorMap wt[2];       // pooling weights hi/lo : [n2 * NT rows (t)][cols (n)], box {64, NT}
};

struct TcArgs {
  const int4* items;       // (alpha, m0, n_tiles, 0) per base, longest first
  int n_base;              // bases; item it = base it % n_base of signal it / n_base, so the
                           // row tiles of one signal's Y run together and share it in L2
  int n_items;             // n_base * B
  int B;
  int passes;              // 1 or 3
  int stages;              // operand pipeline depth (2..8)
  int wstages;             // pooling-weight ring depth (2..kMaxWS)
  int res_kb;              // k-blocks of the resident W tile (RES form)
  int pool_split;          // 1: the 16-frame pooling uses the BF16 hi / lo split
  int n_rows;              // C * n1 (pair rows n_pr in the spin-pair form)
  int pr_phi0;             // spin-pair form: first phi_F pair row
  int nt;                  // frames
  float* P;                // [B][n2][C*n1][nt]
  int n2;
  int* err;                // device status word (0 = ok)
  uint64_t wait_ns;        // budget of every barrier wait (the plan's)
};

// 32 lanes x 32 bits, 32 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int CW>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[CW]) {
  if constexpr (CW == 32) {
    tmem_ld32(taddr, v);
  } else {
    tmem_ld16(taddr, v);
  }
}

// The lambda' range of rate alpha starts at lam_min rounded down to a multiple of 8 (the TMA
// alignment of the W planes) and the MMAs cover it in K = 16 steps, so a rate with 12 rows
// costs one step, not a 32-wide block.  RES = true keeps the item's W tile (every k-block,
// hi and lo) resident in shared memory for all of its column tiles and streams only Y.
template <int NT, int BN, bool RES>
__global__ void __launch_bounds__(kThreads, 1)
k_joint_fwd_tc(const __grid_constant__ TcMaps maps, TcArgs args, DevPlan P) {
  const uint64_t wait_budget = args.wait_ns;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int NH = BN / 64;                           // 64-column halves of a tile
  constexpr int CW = BN / 4;                            // columns per epilogue warp
  const int planes = args.passes == 3 ? 2 : 1;          // hi (+ lo)
  const int S = args.stages, WS = args.wstages;
  constexpr uint32_t kAPlane = kBM * kBK * 2;           // 8 KB, 64-byte swizzle
  constexpr uint32_t kBHalf = kBK * 64 * 2;             // 4 KB: 32 lambda' x 64 samples
  constexpr uint32_t kZHalf = kBM * 64 * 2;             // 16 KB: 128 rows x 64 samples
  constexpr uint32_t kWHalf = NT * 64 * 2;              // NT rows x 64 samples
  const int max_kb = args.res_kb;
  const uint32_t y_bytes = planes * 2 * NH * kBHalf;
  const uint32_t stage_bytes = RES ? y_bytes : planes * 2 * kAPlane + y_bytes;
  uint8_t* sA = sm;                                     // resident W tile (RES)
  uint8_t* sStage = sm + (RES ? planes * 2 * max_kb * kAPlane : 0);
  uint8_t* sZ = sStage + S * stage_bytes;               // planes x NH halves
  uint8_t* sWt = sZ + planes * NH * kZHalf;             // WS buffers x planes x NH halves
  __shared__ uint64_t full_bar[8], empty_bar[8], wfull[kMaxWS], wempty[kMaxWS], tfull, tempty,
      zfull, zempty, d3full, d3free, a_full, a_free, mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int s = 0; s < WS; ++s) {
      mbar_init(&wfull[s], 1);
      mbar_init(&wempty[s], 1);
    }
    mbar_init(&tfull, 1);
    mbar_init(&tempty, kEpiWarps);
    mbar_init(&zfull, kEpiWarps);
    mbar_init(&zempty, 1);
    mbar_init(&d3full, 1);
    mbar_init(&d3free, 4);
    mbar_init(&a_full, 1);
    mbar_init(&a_free, 1);
    mbar_init(&mma_done, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t t_re = tbase, t_im = tbase + BN, t_pool = tbase + 2 * BN;

  auto fail = [&](int code) {
    if (!abort_flag) {
      abort_flag = 1;
      atomicCAS(args.err, 0, code);
    }
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0, ws = 0;
      uint32_t phase = 0, wph = 0, aph = 0;
      // stages / weight buffers with a load in flight, and the parity each one completes
      uint32_t armed = 0, armed_par = 0, armed_w = 0, armed_w_par = 0;
      int armed_a = -1;
      bool ok = true;
      for (int it = blockIdx.x; it < args.n_items && ok && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it % args.n_base];
        const int a = item.x, b = it / args.n_base, m0 = item.y, ntiles = item.z;
        const Rate2 A = P.rates2[a];
        const int lm8 = A.lam_min & ~7;
        const int nkb = (((P.n1 - lm8 + 15) >> 4) + 1) >> 1;
        if (RES) {
          if (!mbar_wait(&a_free, aph ^ 1, wait_budget)) { fail(10); ok = false; break; }
          mbar_arrive_expect_tx(&a_full, planes * 2 * nkb * kAPlane);
          armed_a = (int)aph;
          for (int pl = 0; pl < planes; ++pl)
            for (int part = 0; part < 2; ++part)
              for (int kb = 0; kb < nkb; ++kb)
                tma_load_2d(sA + ((pl * 2 + part) * max_kb + kb) * kAPlane,
                            &maps.w[pl * 2 + part], lm8 + kb * kBK, m0, &a_full);
          aph ^= 1;
        }
        for (int j = 0; j < ntiles && ok; ++j) {
          // operand k-blocks of the tile first, then its pooling weights
          for (int kb = 0; kb < nkb; ++kb) {
            if (!mbar_wait(&empty_bar[stage], phase ^ 1, wait_budget)) { fail(11); ok = false; break; }
            uint8_t* st = sStage + stage * stage_bytes;
            mbar_arrive_expect_tx(&full_bar[stage], stage_bytes);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
            uint8_t* sb = RES ? st : st + planes * 2 * kAPlane;
            for (int pl = 0; pl < planes; ++pl) {
              for (int part = 0; part < 2; ++part) {
                if (!RES)
                  tma_load_2d(st + (pl * 2 + part) * kAPlane, &maps.w[pl * 2 + part],
                              lm8 + kb * kBK, m0, &full_bar[stage]);
                for (int h = 0; h < NH; ++h)
                  tma_load_3d(sb + ((pl * 2 + part) * NH + h) * kBHalf, &maps.y[pl][a],
                              j * BN + h * 64, lm8 + kb * kBK - A.lam_min, 2 * b + part,
                              &full_bar[stage]);
              }
            }
            if (++stage == S) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          if (!mbar_wait(&wempty[ws], wph ^ 1, wait_budget)) { fail(15); ok = false; break; }
          mbar_arrive_expect_tx(&wfull[ws], planes * NH * kWHalf);
          armed_w |= 1u << ws;
          armed_w_par = (armed_w_par & ~(1u << ws)) | (wph << ws);
          for (int pl = 0; pl < planes; ++pl)
            for (int h = 0; h < NH; ++h)
              tma_load_2d(sWt + ((ws * planes + pl) * NH + h) * kWHalf, &maps.wt[pl],
                          j * BN + h * 64, a * NT, &wfull[ws]);
          if (++ws == WS) { ws = 0; wph ^= 1; }
        }
      }
      // never leave the CTA with a copy in flight
      for (int s2 = 0; s2 < S; ++s2)
        if (armed >> s2 & 1) mbar_wait(&full_bar[s2], armed_par >> s2 & 1, wait_budget);
      for (int s2 = 0; s2 < WS; ++s2)
        if (armed_w >> s2 & 1) mbar_wait(&wfull[s2], armed_w_par >> s2 & 1, wait_budget);
      if (armed_a >= 0) mbar_wait(&a_full, (uint32_t)armed_a, wait_budget);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id_pos = instr_desc(kBM, BN, 1, 1, 0, 1, 0);
      const uint32_t id_neg = instr_desc(kBM, BN, 1, 1, 0, 1, 1);
      const uint32_t id_pool = instr_desc(kBM, NT, 1, 1, 0, 0, 0);
      const int npair = args.passes == 3 ? 3 : 1;
      int stage = 0, wq = 0;
      uint32_t phase = 0, tph = 0, zph = 0, wph = 0, d3ph = 0, aph = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < args.n_items && ok && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it % args.n_base];
        const Rate2 A = P.rates2[item.x];
        const int lm8 = A.lam_min & ~7;
        const int nks = (P.n1 - lm8 + 15) >> 4;           // K = 16 steps of the item
        const int nkb = (nks + 1) >> 1;
        const int ntiles = item.z;
        if (RES) {
          if (!mbar_wait(&a_full, aph, wait_budget)) { fail(9); ok = false; break; }
          aph ^= 1;
        }
        for (int j = 0; j <= ntiles && ok; ++j) {
          if (j < ntiles) {
            // the epilogue has loaded the previous tile out of the accumulator
            if (!mbar_wait(&tempty, tph ^ 1, wait_budget)) { fail(12); ok = false; break; }
            tc_fence_after();
            for (int kb = 0; kb < nkb; ++kb) {
              if (!mbar_wait(&full_bar[stage], phase, wait_budget)) { fail(13); ok = false; break; }
              tc_fence_after();
              const uint32_t st = smem_u32(sStage + stage * stage_bytes);
              const uint32_t sb = RES ? st : st + planes * 2 * kAPlane;
              const uint32_t sa = RES ? smem_u32(sA) + kb * kAPlane : st;
              const uint32_t a_stride = RES ? max_kb * kAPlane : kAPlane;   // Re -> Im plane
              const int kss = min(2, nks - 2 * kb);
              for (int ks = 0; ks < kss; ++ks) {
                for (int q = 0; q < npair; ++q) {
                  const int pa = q == 2 ? 1 : 0, pb = q == 1 ? 1 : 0;    // hi.hi, hi.lo, lo.hi
                  const uint32_t ar_a = sa + pa * 2 * a_stride + ks * 32;
                  const uint64_t ar = smem_desc(ar_a, 16, 512, kSw64);
                  const uint64_t ai = smem_desc(ar_a + a_stride, 16, 512, kSw64);
                  const uint32_t br_a = sb + pb * 2 * NH * kBHalf + ks * 2048;
                  const uint64_t br = smem_desc(br_a, kBHalf, 1024, kSw128);
                  const uint64_t bi = smem_desc(br_a + NH * kBHalf, kBHalf, 1024, kSw128);
                  const uint32_t f = (kb | ks | q) ? 1u : 0u;
                  mma_f16(t_re, ar, br, id_pos, f);    // Wr Yr
                  mma_f16(t_re, ai, bi, id_neg, 1u);   // -Wi Yi
                  mma_f16(t_im, ar, bi, id_pos, f);    // Wr Yi
                  mma_f16(t_im, ai, br, id_pos, 1u);   // Wi Yr
                }
              }
              mma_commit(&empty_bar[stage]);
              if (++stage == S) { stage = 0; phase ^= 1; }
            }
            if (!ok) break;
            mma_commit(&tfull);
            tph ^= 1;
          }
          if (j >= 1) {
            // pool the previous tile: D3 += |Z| (128 x BN) . w^T (BN x NT)
            if (!mbar_wait(&zfull, zph, wait_budget)) { fail(16); ok = false; break; }
            if (!mbar_wait(&wfull[wq], wph, wait_budget)) { fail(17); ok = false; break; }
            if (j == 1) {
              if (!mbar_wait(&d3free, d3ph ^ 1, wait_budget)) { fail(18); ok = false; break; }
              d3ph ^= 1;
            }
            tc_fence_after();
            const uint32_t za = smem_u32(sZ);
            const uint32_t wa = smem_u32(sWt + wq * planes * NH * kWHalf);
            for (int ks = 0; ks < BN / 16; ++ks) {
              const uint32_t zo = (ks >> 2) * kZHalf + (ks & 3) * 32;
              const uint32_t wo = (ks >> 2) * kWHalf + (ks & 3) * 32;
              for (int q = 0; q < npair; ++q) {
                const int pa = q == 2 ? 1 : 0, pb = q == 1 ? 1 : 0;
                mma_f16(t_pool, smem_desc(za + pa * NH * kZHalf + zo, 16, 1024, kSw128),
                        smem_desc(wa + pb * NH * kWHalf + wo, 16, 1024, kSw128), id_pool,
                        (j == 1 && ks == 0 && q == 0) ? 0u : 1u);
              }
            }
            mma_commit(&zempty);
            mma_commit(&wempty[wq]);
            zph ^= 1;
            if (++wq == WS) { wq = 0; wph ^= 1; }
          }
        }
        if (!ok) break;
        if (RES) mma_commit(&a_free);
        mma_commit(&d3full);
      }
      mma_commit(&mma_done);
      mbar_wait(&mma_done, 0, wait_budget);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - kEpiWarp0;          // 0..15
    const int quarter = warp & 3;             // TMEM lane quarter this warp may access
    const int cg = ew >> 2;                   // column group: columns [cg CW, cg CW + CW)
    const int row = quarter * 32 + lane;      // tile row
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    // |Z| staging (K-major, 128-byte swizzle): half h = (cg CW) / 64, 16-byte chunk
    // index (cg CW % 64) / 8 + c, swizzled with row & 7
    uint8_t* zrow = sZ + ((cg * CW) >> 6) * kZHalf + row * 128;
    const int chunk0 = ((cg * CW) & 63) >> 3;
    const int sw = row & 7;
    uint32_t tph = 0, zph = 0, d3ph = 0;
    for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
      const int4 item = args.items[it % args.n_base];
      const int a = item.x, b = it / args.n_base, m0 = item.y;
      bool ok = !abort_flag;
      for (int j = 0; j < item.z && ok; ++j) {
        if (!mbar_wait(&tfull, tph, wait_budget)) { fail(14); ok = false; break; }
        tph ^= 1;
        tc_fence_after();
        float re[CW], im[CW];
        tmem_ld_cols<CW>(t_re + lane_off + cg * CW, re);
        tmem_ld_cols<CW>(t_im + lane_off + cg * CW, im);
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty);
        uint32_t hv[CW / 2], lv[CW / 2];
#pragma unroll
        for (int i = 0; i < CW / 2; ++i) {
          // element pairs (2i, 2i + 1) in packed FP32 operations
          const float2 r2 = make_float2(re[2 * i], re[2 * i + 1]);
          const float2 i2 = make_float2(im[2 * i], im[2 * i + 1]);
          const float2 m2 = __ffma2_rn(r2, r2, __fmul2_rn(i2, i2));
          const float2 mv = make_float2(sqrt_approx(m2.x), sqrt_approx(m2.y));
          __nv_bfloat162 h = __floats2bfloat162_rn(mv.x, mv.y);
          const float2 d = fsub2(mv, __bfloat1622float2(h));
          __nv_bfloat162 l = __floats2bfloat162_rn(d.x, d.y);
          hv[i] = *reinterpret_cast<uint32_t*>(&h);
          lv[i] = *reinterpret_cast<uint32_t*>(&l);
        }
        if (!mbar_wait(&zempty, zph ^ 1, wait_budget)) { fail(19); ok = false; break; }
        zph ^= 1;
#pragma unroll
        for (int c = 0; c < CW / 8; ++c) {
          const int pos = ((chunk0 + c) ^ sw) * 16;
          *reinterpret_cast<uint4*>(zrow + pos) =
              make_uint4(hv[4 * c], hv[4 * c + 1], hv[4 * c + 2], hv[4 * c + 3]);
          if (planes == 2)
            *reinterpret_cast<uint4*>(zrow + NH * kZHalf + pos) =
                make_uint4(lv[4 * c], lv[4 * c + 1], lv[4 * c + 2], lv[4 * c + 3]);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&zfull);
      }
      if (!ok) break;
      if (cg != 0) continue;                  // one warp per lane quarter reads the pooled rows
      if (!mbar_wait(&d3full, d3ph, wait_budget)) { fail(20); break; }
      d3ph ^= 1;
      tc_fence_after();
      const int r = m0 + row;
      float* out = args.P + (((size_t)b * args.n2 + a) * args.n_rows + r) * args.nt;
#pragma unroll
      for (int c = 0; c < NT; c += 16) {
        float v[16];
        tmem_ld16(t_pool + lane_off + c, v);
        tmem_wait_ld();
        if (r < args.n_rows) {
          if ((args.nt & 3) == 0) {
#pragma unroll
            for (int t = 0; t < 16; t += 4)
              if (c + t < args.nt)
                *reinterpret_cast<float4*>(out + c + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
          } else {
#pragma unroll
            for (int t = 0; t < 16; ++t)
              if (c + t < args.nt) out[c + t] = v[t];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&d3free);
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// ------------------------------------------------------------------ 16-frame form
// With 16 pooled frames the phi_T pooling runs in the epilogue warps on the warp-level
// tensor-core path (mma.sync m16n8k16, BF16 in, FP32 accumulate), which leaves all 512 TMEM
// columns to two 128 x 128 complex accumulators: the next tile's product is issued while the
// epilogue drains the previous one, and no pooling MMA sits between them.
//
// Each epilogue warp owns 32 rows (its TMEM lane quarter) x 32 columns of a tile.  Per
// 16-column step it stages |Z| (hi, and lo for the split) in a private 32 x 16 BF16 block,
// loads mma.sync fragments with ldmatrix and accumulates P[row, t] = sum_n |Z| w[n, t] in
// registers over every tile of the item; at the end the four column groups of a quarter
// are summed through shared memory in a fixed order.
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}
__device__ __forceinline__ void hmma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                          uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Launched with TF = true: TF32 operands (FP32 W and Y planes, kind::tf32 MMAs of K = 8, one
// pass); the pooling then keeps the BF16 hi / lo split.  BF16 planes at 16 frames take the
// spin-pair form below instead.
template <bool RES, bool TF>
__global__ void __launch_bounds__(kThreads, 1)
k_joint_fwd_tc16(const __grid_constant__ TcMaps maps, TcArgs args, DevPlan P) {
  const uint64_t wait_budget = args.wait_ns;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int NT = 16, BN = 128, NH = 2;
  // contraction planes (hi, + lo for the BF16 split) and pooling planes (|Z| and w: hi, + lo)
  const int planes = TF ? 1 : (args.passes == 3 ? 2 : 1);
  const int pplanes = args.pool_split ? 2 : 1;
  const int S = args.stages, WS = args.wstages;
  constexpr uint32_t kAPlane = TF ? kBM * kBK * 4 : kBM * kBK * 2;   // 16 KB SW128 / 8 KB SW64
  constexpr int NYA = TF ? 4 : 2;                       // Y atoms per part: 32 / 64 samples wide
  constexpr int kYAW = BN / NYA;
  constexpr uint32_t kBHalf = 4096;                     // one Y atom: 32 lambda' x 128 bytes
  constexpr uint32_t kWHalf = NT * 64 * 2;              // 2 KB: 16 frames x 64 samples
  constexpr uint32_t kStg = 32 * 16 * 2;                // 1 KB: a warp's 32 x 16 |Z| block
  const int max_kb = args.res_kb;
  const uint32_t y_bytes = planes * 2 * NYA * kBHalf;
  const uint32_t stage_bytes = RES ? y_bytes : planes * 2 * kAPlane + y_bytes;
  uint8_t* sA = sm;
  uint8_t* sStage = sm + (RES ? planes * 2 * max_kb * kAPlane : 0);
  uint8_t* sWt = sStage + S * stage_bytes;              // WS x NH halves x pplanes (hi, lo adjacent)
  uint8_t* sStg = sWt + WS * NH * pplanes * kWHalf;     // 16 warps x pplanes x 1 KB
  float* sRed = (float*)(sStg + kEpiWarps * pplanes * kStg);   // [4 groups][128 rows][16]
  __shared__ uint64_t full_bar[8], empty_bar[8], wfull[kMaxWS], wempty[kMaxWS], tfull[2],
      tempty[2], red_full[4], red_free[4], sfull[4], sfree[4], a_full, a_free, mma_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int s = 0; s < WS; ++s) {
      mbar_init(&wfull[s], 1);
      mbar_init(&wempty[s], kEpiWarps);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], kEpiWarps);
    }
    for (int q = 0; q < 4; ++q) {
      mbar_init(&red_full[q], 4);
      mbar_init(&red_free[q], 1);
      mbar_init(&sfull[q], 4);
      mbar_init(&sfree[q], 4);
    }
    mbar_init(&a_full, 1);
    mbar_init(&a_free, 1);
    mbar_init(&mma_done, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;

  auto fail = [&](int code) {
    if (!abort_flag) {
      abort_flag = 1;
      atomicCAS(args.err, 0, code);
    }
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0, ws = 0;
      uint32_t phase = 0, wph = 0, aph = 0;
      uint32_t armed = 0, armed_par = 0, armed_w = 0, armed_w_par = 0;
      int armed_a = -1;
      bool ok = true;
      for (int it = blockIdx.x; it < args.n_items && ok && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it % args.n_base];
        const int a = item.x, b = it / args.n_base, m0 = item.y, ntiles = item.z;
        const Rate2 A = P.rates2[a];
        const int lm8 = A.lam_min & ~7;
        const int nkb = (((P.n1 - lm8 + 15) >> 4) + 1) >> 1;
        if (RES) {
          if (!mbar_wait(&a_free, aph ^ 1, wait_budget)) { fail(10); ok = false; break; }
          mbar_arrive_expect_tx(&a_full, planes * 2 * nkb * kAPlane);
          armed_a = (int)aph;
          for (int pl = 0; pl < planes; ++pl)
            for (int part = 0; part < 2; ++part)
              for (int kb = 0; kb < nkb; ++kb)
                tma_load_2d(sA + ((pl * 2 + part) * max_kb + kb) * kAPlane,
                            &maps.w[pl * 2 + part], lm8 + kb * kBK, m0, &a_full);
          aph ^= 1;
        }
        for (int j = 0; j < ntiles && ok; ++j) {
          for (int kb = 0; kb < nkb; ++kb) {
            if (!mbar_wait(&empty_bar[stage], phase ^ 1, wait_budget)) { fail(11); ok = false; break; }
            uint8_t* st = sStage + stage * stage_bytes;
            mbar_arrive_expect_tx(&full_bar[stage], stage_bytes);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
            uint8_t* sb = RES ? st : st + planes * 2 * kAPlane;
            for (int pl = 0; pl < planes; ++pl) {
              for (int part = 0; part < 2; ++part) {
                if (!RES)
                  tma_load_2d(st + (pl * 2 + part) * kAPlane, &maps.w[pl * 2 + part],
                              lm8 + kb * kBK, m0, &full_bar[stage]);
                if (TF) {
                  // Y^T [n][lambda' - lm8]: one 128-sample x 32-lambda' K-major box per part
                  tma_load_3d(sb + (pl * 2 + part) * NYA * kBHalf, &maps.y[pl][a], kb * kBK,
                              j * BN, 2 * b + part, &full_bar[stage]);
                } else {
                  for (int h = 0; h < NYA; ++h)
                    tma_load_3d(sb + ((pl * 2 + part) * NYA + h) * kBHalf, &maps.y[pl][a],
                                j * BN + h * kYAW, lm8 + kb * kBK - A.lam_min, 2 * b + part,
                                &full_bar[stage]);
                }
              }
            }
            if (++stage == S) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          if (!mbar_wait(&wempty[ws], wph ^ 1, wait_budget)) { fail(15); ok = false; break; }
          mbar_arrive_expect_tx(&wfull[ws], pplanes * NH * kWHalf);
          armed_w |= 1u << ws;
          armed_w_par = (armed_w_par & ~(1u << ws)) | (wph << ws);
          for (int h = 0; h < NH; ++h)
            for (int pl = 0; pl < pplanes; ++pl)
              tma_load_2d(sWt + ((ws * NH + h) * pplanes + pl) * kWHalf, &maps.wt[pl],
                          j * BN + h * 64, a * NT, &wfull[ws]);
          if (++ws == WS) { ws = 0; wph ^= 1; }
        }
      }
      for (int s2 = 0; s2 < S; ++s2)
        if (armed >> s2 & 1) mbar_wait(&full_bar[s2], armed_par >> s2 & 1, wait_budget);
      for (int s2 = 0; s2 < WS; ++s2)
        if (armed_w >> s2 & 1) mbar_wait(&wfull[s2], armed_w_par >> s2 & 1, wait_budget);
      if (armed_a >= 0) mbar_wait(&a_full, (uint32_t)armed_a, wait_budget);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t kFmt = TF ? 2 : 1;
      const uint32_t id_pos = instr_desc(kBM, BN, kFmt, kFmt, 0, TF ? 0 : 1, 0);
      const uint32_t id_neg = instr_desc(kBM, BN, kFmt, kFmt, 0, TF ? 0 : 1, 1);
      const int npair = (!TF && args.passes == 3) ? 3 : 1;
      int stage = 0, acc = 0;
      uint32_t phase = 0, acc_ph = 0, aph = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < args.n_items && ok && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it % args.n_base];
        const Rate2 A = P.rates2[item.x];
        const int lm8 = A.lam_min & ~7;
        // K steps of the item: 16 lambda' (BF16) or 8 (TF32); 32 lambda' per k-block
        constexpr int kKS = TF ? 8 : 16, kSPB = kBK / kKS;
        const int nks = (P.n1 - lm8 + kKS - 1) / kKS;
        const int nkb = (nks + kSPB - 1) / kSPB;
        if (RES) {
          if (!mbar_wait(&a_full, aph, wait_budget)) { fail(9); ok = false; break; }
          aph ^= 1;
        }
        for (int j = 0; j < item.z && ok; ++j) {
          if (!mbar_wait(&tempty[acc], acc_ph ^ 1, wait_budget)) { fail(12); ok = false; break; }
          tc_fence_after();
          const uint32_t t_re = tbase + acc * 256, t_im = t_re + 128;
          for (int kb = 0; kb < nkb; ++kb) {
            if (!mbar_wait(&full_bar[stage], phase, wait_budget)) { fail(13); ok = false; break; }
            tc_fence_after();
            const uint32_t st = smem_u32(sStage + stage * stage_bytes);
            const uint32_t sb = RES ? st : st + planes * 2 * kAPlane;
            const uint32_t sa = RES ? smem_u32(sA) + kb * kAPlane : st;
            const uint32_t a_stride = RES ? max_kb * kAPlane : kAPlane;
            const int kss = min(kSPB, nks - kSPB * kb);
            for (int ks = 0; ks < kss; ++ks) {
              for (int q = 0; q < npair; ++q) {
                const int pa = q == 2 ? 1 : 0, pb = q == 1 ? 1 : 0;
                // A: K-major rows of 32 lambda' (64-byte swizzle for BF16, 128 for FP32);
                // B: MN-major atoms of 128 bytes, K step = 16 (BF16) or 8 (TF32) rows
                const uint32_t ar_a = sa + pa * 2 * a_stride + ks * 32;
                const uint64_t ar = smem_desc(ar_a, 16, TF ? 1024 : 512, TF ? kSw128 : kSw64);
                const uint64_t ai = smem_desc(ar_a + a_stride, 16, TF ? 1024 : 512, TF ? kSw128 : kSw64);
                // B for TF32: K-major [128 samples][32 lambda'], +32 bytes per K = 8 step
                const uint32_t br_a = sb + pb * 2 * NYA * kBHalf + (TF ? ks * 32 : ks * kKS * 128);
                const uint64_t br = smem_desc(br_a, TF ? 16 : kBHalf, 1024, kSw128);
                const uint64_t bi = smem_desc(br_a + NYA * kBHalf, TF ? 16 : kBHalf, 1024, kSw128);
                const uint32_t f = (kb | ks | q) ? 1u : 0u;
                if (TF) {
                  mma_tf32(t_re, ar, br, id_pos, f);    // Wr Yr
                  mma_tf32(t_re, ai, bi, id_neg, 1u);   // -Wi Yi
                  mma_tf32(t_im, ar, bi, id_pos, f);    // Wr Yi
                  mma_tf32(t_im, ai, br, id_pos, 1u);   // Wi Yr
                } else {
                  mma_f16(t_re, ar, br, id_pos, f);
                  mma_f16(t_re, ai, bi, id_neg, 1u);
                  mma_f16(t_im, ar, bi, id_pos, f);
                  mma_f16(t_im, ai, br, id_pos, 1u);
                }
              }
            }
            mma_commit(&empty_bar[stage]);
            if (++stage == S) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(&tfull[acc]);
          if (++acc == 2) { acc = 0; acc_ph ^= 1; }
        }
        if (!ok) break;
        if (RES) mma_commit(&a_free);
      }
      mma_commit(&mma_done);
      mbar_wait(&mma_done, 0, wait_budget);
    }
  } else {
    // ------------------------------------------------------------ epilogue + pooling
    const int ew = warp - kEpiWarp0;          // 0..15
    const int quarter = warp & 3;
    const int cg = ew >> 2;                   // columns [32 cg, 32 cg + 32) of a tile
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int g = lane >> 2, t4 = lane & 3;
    // staging block: row = lane, two 16-byte chunks, chunk ^= (row >> 2) & 1
    uint8_t* stg = sStg + ew * pplanes * kStg;
    const uint32_t stg_u = smem_u32(stg);
    uint8_t* my_row = stg + lane * 32;
    const int my_sw = (lane >> 2) & 1;
    // ldmatrix row addresses: A (16 x 16 block mt): row 16 mt + (lane & 15), chunk lane >> 4
    uint32_t a_addr[2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r = 16 * mt + (lane & 15);
      a_addr[mt] = stg_u + r * 32 + (((lane >> 4) ^ ((r >> 2) & 1)) << 4);
    }
    // B (w tile, [t][n] rows of 128 bytes, 128-byte swizzle): t = 8 (m >> 1) + (lane & 7),
    // 8-sample chunk of the step + (m & 1), with m = lane >> 3
    const int bt = 8 * (lane >> 4) + (lane & 7);
    const int bk = (lane >> 3) & 1;
    int acc = 0, ws = 0;
    uint32_t acc_ph = 0, wph = 0, rf_ph = 0, rfree_ph = 0;
    for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
      const int4 item = args.items[it % args.n_base];
      const int a = item.x, b = it / args.n_base, m0 = item.y;
      bool ok = !abort_flag;
      float c[2][2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int e = 0; e < 4; ++e) c[i][k][e] = 0.f;
      for (int j = 0; j < item.z && ok; ++j) {
        if (!mbar_wait(&tfull[acc], acc_ph, wait_budget)) { fail(14); ok = false; break; }
        tc_fence_after();
        if (!mbar_wait(&wfull[ws], wph, wait_budget)) { fail(19); ok = false; break; }
        const uint32_t t_col = tbase + acc * 256 + lane_off + cg * 32;
        const uint32_t w_u = smem_u32(sWt + (ws * NH + (cg >> 1)) * pplanes * kWHalf);
#pragma unroll
        for (int sub = 0; sub < 2; ++sub) {
          float re[16], im[16];
          tmem_ld16(t_col + sub * 16, re);
          tmem_ld16(t_col + 128 + sub * 16, im);
          tmem_wait_ld();
          if (sub == 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
          }
          uint32_t hv[8], lv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            // element pairs (2i, 2i + 1) in packed FP32 operations
            const float2 r2 = make_float2(re[2 * i], re[2 * i + 1]);
            const float2 i2 = make_float2(im[2 * i], im[2 * i + 1]);
            const float2 m2 = __ffma2_rn(r2, r2, __fmul2_rn(i2, i2));
            const float2 mv = make_float2(sqrt_approx(m2.x), sqrt_approx(m2.y));
            __nv_bfloat162 h = __floats2bfloat162_rn(mv.x, mv.y);
            const float2 d = fsub2(mv, __bfloat1622float2(h));
            __nv_bfloat162 l = __floats2bfloat162_rn(d.x, d.y);
            hv[i] = *reinterpret_cast<uint32_t*>(&h);
            lv[i] = *reinterpret_cast<uint32_t*>(&l);
          }
          __syncwarp();   // the previous step's fragment loads are done
#pragma unroll
          for (int ch = 0; ch < 2; ++ch) {
            const int pos = (ch ^ my_sw) * 16;
            *reinterpret_cast<uint4*>(my_row + pos) =
                make_uint4(hv[4 * ch], hv[4 * ch + 1], hv[4 * ch + 2], hv[4 * ch + 3]);
            if (pplanes == 2)
              *reinterpret_cast<uint4*>(my_row + kStg + pos) =
                  make_uint4(lv[4 * ch], lv[4 * ch + 1], lv[4 * ch + 2], lv[4 * ch + 3]);
          }
          __syncwarp();
          // B fragments: w[t][n] for n in this step's 16 columns of the 64-column half
          const int chunk = (((cg & 1) * 32 + sub * 16) >> 3) + bk;
          const uint32_t b_off = bt * 128 + ((chunk ^ (bt & 7)) << 4);
          uint32_t bh[4], ah[2][4];
          ldsm_x4(w_u + b_off, bh);
          ldsm_x4(a_addr[0], ah[0]);
          ldsm_x4(a_addr[1], ah[1]);
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            hmma16816(c[mt][0], ah[mt], bh[0], bh[1]);
            hmma16816(c[mt][1], ah[mt], bh[2], bh[3]);
          }
          if (pplanes == 2) {
            uint32_t bl[4], al[2][4];
            ldsm_x4(w_u + kWHalf + b_off, bl);
            ldsm_x4(a_addr[0] + kStg, al[0]);
            ldsm_x4(a_addr[1] + kStg, al[1]);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
              hmma16816(c[mt][0], ah[mt], bl[0], bl[1]);   // hi . lo
              hmma16816(c[mt][1], ah[mt], bl[2], bl[3]);
              hmma16816(c[mt][0], al[mt], bh[0], bh[1]);   // lo . hi
              hmma16816(c[mt][1], al[mt], bh[2], bh[3]);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&wempty[ws]);
        if (++ws == WS) { ws = 0; wph ^= 1; }
        if (++acc == 2) { acc = 0; acc_ph ^= 1; }
      }
      if (!ok) break;
      // sum the four column groups of this lane quarter in a fixed order
      if (cg != 0) {
        if (!mbar_wait(&red_free[quarter], rfree_ph ^ 1, wait_budget)) { fail(21); break; }
        rfree_ph ^= 1;
      }
      float* red = sRed + (cg * 128 + quarter * 32) * NT;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int r = 16 * mt + g, t = 8 * nt + 2 * t4;
          *reinterpret_cast<float2*>(red + r * NT + t) = make_float2(c[mt][nt][0], c[mt][nt][1]);
          *reinterpret_cast<float2*>(red + (r + 8) * NT + t) = make_float2(c[mt][nt][2], c[mt][nt][3]);
        }
      __syncwarp();
      if (lane == 0) mbar_arrive(&red_full[quarter]);
      if (cg == 0) {
        if (!mbar_wait(&red_full[quarter], rf_ph, wait_budget)) { fail(20); break; }
        rf_ph ^= 1;
        const int r = m0 + quarter * 32 + lane;
        float s[NT];
#pragma unroll
        for (int t = 0; t < NT; ++t) s[t] = 0.f;
#pragma unroll
        for (int gq = 0; gq < 4; ++gq) {
          const float* src = sRed + (gq * 128 + quarter * 32 + lane) * NT;
#pragma unroll
          for (int t = 0; t < NT; t += 4) {
            const float4 v = *reinterpret_cast<const float4*>(src + t);
            s[t] += v.x; s[t + 1] += v.y; s[t + 2] += v.z; s[t + 3] += v.w;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&red_free[quarter]);
        if (r < args.n_rows) {
          float* out = args.P + (((size_t)b * args.n2 + a) * args.n_rows + r) * args.nt;
          if (args.nt == NT) {
#pragma unroll
            for (int t = 0; t < NT; t += 4)
              *reinterpret_cast<float4*>(out + t) = make_float4(s[t], s[t + 1], s[t + 2], s[t + 3]);
          } else {
#pragma unroll
            for (int t = 0; t < NT; ++t)
              if (t < args.nt) out[t] = s[t];
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// ------------------------------------------------------------------ spin-pair form
// The spin-down log-frequency filters are the complex conjugates of the spin-up ones
// (psi_{beta,-1}-hat(omega) = psi_{beta,+1}-hat(-omega) with a real spectrum that vanishes at
// DC and Nyquist), so for a pair of rows (up c, down c + n_fr) with W_up = Wr + i Wi:
//   Z_up = (Wr Yr - Wi Yi) + i (Wr Yi + Wi Yr),   Z_down = (Wr Yr + Wi Yi) + i (Wr Yi - Wi Yr).
// The four real products come from two MMAs per K step over a 64-sample tile with
// B = [Yr | Yi] (N = 128): [P1 | P3] = Wr [Yr | Yi], [P4 | P2] = Wi [Yr | Yi]; the epilogue
// forms both channels.  That halves the contraction's MMAs against the channel-row form.
// Rows are pair rows r = p n1 + lambda for the spin pairs p < n_fr, then zero rows up to the
// next multiple of 32, then the n1 rows of the phi_F branch (real W, only its "up" output is
// written).
// The phi_T pooling runs on the tensor cores too (an earlier form pooled with mma.sync in the
// epilogue, at a quarter of the tcgen05 rate).  The epilogue stages |Z| (BF16 hi, lo for the
// FP32-grade split) of both spins in tensor memory as an MMA A operand (row r in lane r, two
// samples per 32-bit column: 32 columns per spin and plane), and a second issuing thread
// accumulates D_spin[row][f] += |Z|[row][n] [W_hi | W_lo][f][n] over the item's tiles into TMEM
// (N = NT per weight plane: frames of W_hi, then of W_lo; both |Z| planes accumulate into the
// same D, so D[f] + D[NT + f] = (Z_hi + Z_lo)(W_hi + W_lo)).  Staging |Z| in tensor memory
// keeps its stores and the pooling MMAs' A reads off the shared memory, whose bandwidth the
// product MMAs (8 KB per M = 128, N = 128, K = 16 step) already fill.  The TMEM holds one
// 256-column product accumulator, the two pooling accumulators and the staged |Z|, so the
// product of tile j + 1 starts once the epilogue has loaded tile j.  At an item's end warp
// (quarter, cg) reads spin cg >> 1, frames [NT / 2 (cg & 1), +NT / 2) of its 32 rows and
// writes them.
constexpr int kTpThreads = 32 * 19;   // producer, product issuer, 16 epilogue warps, pooling issuer
constexpr int kTpWarpPool = 18;

template <bool RES, int PS, int NT>
__global__ void __launch_bounds__(kTpThreads, 1)
k_joint_fwd_tp(const __grid_constant__ TcMaps maps, TcArgs args, DevPlan P) {
  static_assert(NT == 16 || NT == 32, "pooled frames");
  const uint64_t wait_budget = args.wait_ns;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int BN = 64;
  constexpr int NP = PS * NT;                            // pooling N (frames of W_hi [, W_lo])
  const int planes = args.passes == 3 ? 2 : 1;
  const int S = args.stages, WS = args.wstages;
  constexpr uint32_t kAPlane = kBM * kBK * 2;            // 8 KB: 128 rows x 32 lambda', SW64
  constexpr uint32_t kYAtom = 4096;                      // 32 lambda' x 64 samples, SW128
  constexpr uint32_t kWHalf = NT * 64 * 2;               // one weight plane: NT frames x 64 samples
  const int max_kb = args.res_kb;
  const uint32_t y_bytes = planes * 2 * kYAtom;          // per plane [Yr atom | Yi atom]
  const uint32_t stage_bytes = RES ? y_bytes : planes * 2 * kAPlane + y_bytes;
  uint8_t* sA = sm;
  uint8_t* sStage = sm + (RES ? planes * 2 * max_kb * kAPlane : 0);
  uint8_t* sWt = sStage + S * stage_bytes;               // WS slots of [W_hi plane][W_lo plane]
  __shared__ uint64_t full_bar[8], empty_bar[8], wfull[kMaxWS], wempty[kMaxWS], tfull, tempty,
      sfull, sfree, dfull, dfree, a_full, a_free, mma_done, pool_done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int s = 0; s < WS; ++s) {
      mbar_init(&wfull[s], 1);
      mbar_init(&wempty[s], 1);
    }
    mbar_init(&tfull, 1);
    mbar_init(&tempty, kEpiWarps);
    mbar_init(&sfull, kEpiWarps);
    mbar_init(&sfree, 1);
    mbar_init(&dfull, 1);
    mbar_init(&dfree, kEpiWarps);
    mbar_init(&a_full, 1);
    mbar_init(&a_free, 1);
    mbar_init(&mma_done, 1);
    mbar_init(&pool_done, 1);
    fence_barrier_init();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base, 512);
    tmem_relinquish();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t t_pool = tbase + 256;                   // [spin] NP columns each
  const uint32_t t_z = t_pool + 2 * NP;                  // [spin][plane] 32 columns of |Z|
  static_assert(256 + 2 * NP + 2 * PS * 32 <= 512, "TMEM columns");

  auto fail = [&](int code) {
    if (!abort_flag) {
      abort_flag = 1;
      atomicCAS(args.err, 0, code);
    }
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int stage = 0, ws = 0;
      uint32_t phase = 0, wph = 0, aph = 0;
      uint32_t armed = 0, armed_par = 0, armed_w = 0, armed_w_par = 0;
      int armed_a = -1;
      bool ok = true;
      for (int it = blockIdx.x; it < args.n_items && ok && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it % args.n_base];
        const int a = item.x, b = it / args.n_base, m0 = item.y, ntiles = item.z;
        const Rate2 A = P.rates2[a];
        const int lm8 = A.lam_min & ~7;
        const int nkb = (((P.n1 - lm8 + 15) >> 4) + 1) >> 1;
        if (RES) {
          if (!mbar_wait(&a_free, aph ^ 1, wait_budget)) { fail(30); ok = false; break; }
          mbar_arrive_expect_tx(&a_full, planes * 2 * nkb * kAPlane);
          armed_a = (int)aph;
          for (int pl = 0; pl < planes; ++pl)
            for (int part = 0; part < 2; ++part)
              for (int kb = 0; kb < nkb; ++kb)
                tma_load_2d(sA + ((pl * 2 + part) * max_kb + kb) * kAPlane,
                            &maps.w[pl * 2 + part], lm8 + kb * kBK, m0, &a_full);
          aph ^= 1;
        }
        for (int j = 0; j < ntiles && ok; ++j) {
          for (int kb = 0; kb < nkb; ++kb) {
            if (!mbar_wait(&empty_bar[stage], phase ^ 1, wait_budget)) { fail(31); ok = false; break; }
            uint8_t* st = sStage + stage * stage_bytes;
            mbar_arrive_expect_tx(&full_bar[stage], stage_bytes);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
            uint8_t* sb = RES ? st : st + planes * 2 * kAPlane;
            for (int pl = 0; pl < planes; ++pl) {
              for (int part = 0; part < 2; ++part) {
                if (!RES)
                  tma_load_2d(st + (pl * 2 + part) * kAPlane, &maps.w[pl * 2 + part],
                              lm8 + kb * kBK, m0, &full_bar[stage]);
                tma_load_3d(sb + (pl * 2 + part) * kYAtom, &maps.y[pl][a], j * BN,
                            lm8 + kb * kBK - A.lam_min, 2 * b + part, &full_bar[stage]);
              }
            }
            if (++stage == S) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          if (!mbar_wait(&wempty[ws], wph ^ 1, wait_budget)) { fail(32); ok = false; break; }
          mbar_arrive_expect_tx(&wfull[ws], PS * kWHalf);
          armed_w |= 1u << ws;
          armed_w_par = (armed_w_par & ~(1u << ws)) | (wph << ws);
          for (int pl = 0; pl < PS; ++pl)
            tma_load_2d(sWt + (ws * PS + pl) * kWHalf, &maps.wt[pl], j * BN, a * NT, &wfull[ws]);
          if (++ws == WS) { ws = 0; wph ^= 1; }
        }
      }
      for (int s2 = 0; s2 < S; ++s2)
        if (armed >> s2 & 1) mbar_wait(&full_bar[s2], armed_par >> s2 & 1, wait_budget);
      for (int s2 = 0; s2 < WS; ++s2)
        if (armed_w >> s2 & 1) mbar_wait(&wfull[s2], armed_w_par >> s2 & 1, wait_budget);
      if (armed_a >= 0) mbar_wait(&a_full, (uint32_t)armed_a, wait_budget);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ product issuer
    if (lane == 0) {
      const uint32_t id = instr_desc(kBM, 128, 1, 1, 0, 1, 0);
      const int npair = args.passes == 3 ? 3 : 1;
      int stage = 0;
      uint32_t phase = 0, tph = 0, aph = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < args.n_items && ok && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it % args.n_base];
        const Rate2 A = P.rates2[item.x];
        const int lm8 = A.lam_min & ~7;
        const int nks = (P.n1 - lm8 + 15) / 16;
        const int nkb = (nks + 1) / 2;
        if (RES) {
          if (!mbar_wait(&a_full, aph, wait_budget)) { fail(33); ok = false; break; }
          aph ^= 1;
        }
        for (int j = 0; j < item.z && ok; ++j) {
          if (!mbar_wait(&tempty, tph ^ 1, wait_budget)) { fail(34); ok = false; break; }
          tph ^= 1;
          tc_fence_after();
          const uint32_t t_a = tbase, t_b = tbase + 128;
          for (int kb = 0; kb < nkb; ++kb) {
            if (!mbar_wait(&full_bar[stage], phase, wait_budget)) { fail(35); ok = false; break; }
            tc_fence_after();
            const uint32_t st = smem_u32(sStage + stage * stage_bytes);
            const uint32_t sb = RES ? st : st + planes * 2 * kAPlane;
            const uint32_t sa = RES ? smem_u32(sA) + kb * kAPlane : st;
            const uint32_t a_stride = RES ? max_kb * kAPlane : kAPlane;
            const int kss = min(2, nks - 2 * kb);
            const uint64_t dA = smem_desc(sa, 16, 512, kSw64);
            const uint64_t dB = smem_desc(sb, kYAtom, 1024, kSw128);
            const uint32_t as4 = a_stride >> 4;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              if (ks < kss) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                  if (q < npair) {
                    const int pa = q == 2 ? 1 : 0, pb = q == 1 ? 1 : 0;
                    const uint64_t ar = dA + (uint64_t)(pa * 2 * as4 + ks * 2);
                    const uint64_t ai = ar + as4;
                    const uint64_t bd = dB + (uint64_t)(pb * 2 * (kYAtom >> 4) + ks * 128);
                    const uint32_t f = (kb | ks | q) ? 1u : 0u;
                    mma_f16(t_a, ar, bd, id, f);    // [P1 | P3] = Wr [Yr | Yi]
                    mma_f16(t_b, ai, bd, id, f);    // [P4 | P2] = Wi [Yr | Yi]
                  }
                }
              }
            }
            mma_commit(&empty_bar[stage]);
            if (++stage == S) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(&tfull);
        }
        if (!ok) break;
        if (RES) mma_commit(&a_free);
      }
      mma_commit(&mma_done);
      mbar_wait(&mma_done, 0, wait_budget);
    }
  } else if (warp == kTpWarpPool) {
    // ------------------------------------------------------------ pooling issuer
    if (lane == 0) {
      // A = |Z| [128 rows][64 samples] in tensor memory, B = [W_hi ; W_lo] [NP frames][64
      // samples] K-major with 128-byte rows; a K step is 16 samples
      const uint32_t idp = instr_desc(kBM, NP, 1, 1, 0, 0, 0);
      int ws = 0;
      uint32_t sph = 0, wph = 0, dph = 0;
      bool ok = true;
      for (int it = blockIdx.x; it < args.n_items && ok && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it % args.n_base];
        // the epilogue has read the previous item's accumulators
        if (!mbar_wait(&dfree, dph ^ 1, wait_budget)) { fail(36); ok = false; break; }
        dph ^= 1;
        for (int j = 0; j < item.z && ok; ++j) {
          if (!mbar_wait(&sfull, sph, wait_budget)) { fail(37); ok = false; break; }
          sph ^= 1;
          if (!mbar_wait(&wfull[ws], wph, wait_budget)) { fail(38); ok = false; break; }
          tc_fence_after();
          const uint64_t dW = smem_desc(smem_u32(sWt + ws * PS * kWHalf), 16, 1024, kSw128);
#pragma unroll
          for (int d = 0; d < 2; ++d)
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
              for (int pa = 0; pa < PS; ++pa) {
                // A: samples [16 k, 16 k + 16) of |Z| (spin d, plane pa) in tensor memory
                const uint64_t bw = dW + (uint64_t)((k * 32) >> 4);
                mma_f16_ta(t_pool + d * NP, t_z + (d * PS + pa) * 32 + k * 8, bw, idp,
                           (j | k | pa) ? 1u : 0u);
              }
          mma_commit(&sfree);
          mma_commit(&wempty[ws]);
          if (++ws == WS) { ws = 0; wph ^= 1; }
        }
        if (!ok) break;
        mma_commit(&dfull);
      }
      mma_commit(&pool_done);
      mbar_wait(&pool_done, 0, wait_budget);
    }
  } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + kEpiWarps) {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - kEpiWarp0;          // 0..15
    const int quarter = warp & 3;
    const int cg = ew >> 2;                   // samples [16 cg, 16 cg + 16) of the tile
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int row = quarter * 32 + lane;      // row of the 128-row block (TMEM lane)
    // this warp's |Z| columns: samples [16 cg, 16 cg + 16) of each (spin, plane) block
    const uint32_t t_zw = t_z + lane_off + cg * 8;
    uint32_t tph = 0, sph = 0, dph = 0;
    for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
      const int4 item = args.items[it % args.n_base];
      const int a = item.x, b = it / args.n_base, m0 = item.y;
      bool ok = !abort_flag;
      for (int j = 0; j < item.z && ok; ++j) {
        if (!mbar_wait(&tfull, tph, wait_budget)) { fail(39); ok = false; break; }
        tph ^= 1;
        tc_fence_after();
        const uint32_t t_col = tbase + lane_off + cg * 16;
        uint32_t hv[2][2][4], lv[2][2][4];     // [h8][spin][4 bf16x2]
        // the whole accumulator share (four products x 16 samples) is loaded before it is
        // released, so the next tile's product waits for the loads alone
        uint32_t q1[2][8], q3[2][8], q4[2][8], q2[2][8];
#pragma unroll
        for (int h8 = 0; h8 < 2; ++h8) {
          tmem_ld8u(t_col + h8 * 8, q1[h8]);
          tmem_ld8u(t_col + h8 * 8 + 64, q3[h8]);
          tmem_ld8u(t_col + h8 * 8 + 128, q4[h8]);
          tmem_ld8u(t_col + h8 * 8 + 192, q2[h8]);
        }
        tmem_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty);
#pragma unroll
        for (int h8 = 0; h8 < 2; ++h8) {
          const uint32_t* p1 = q1[h8];
          const uint32_t* p3 = q3[h8];
          const uint32_t* p4 = q4[h8];
          const uint32_t* p2 = q2[h8];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            // samples' element pairs (2i, 2i + 1) in packed FP32 operations
            const float2 x1 = u2f2(p1[2 * i], p1[2 * i + 1]), x2 = u2f2(p2[2 * i], p2[2 * i + 1]);
            const float2 x3 = u2f2(p3[2 * i], p3[2 * i + 1]), x4 = u2f2(p4[2 * i], p4[2 * i + 1]);
            const float2 ru = fsub2(x1, x2), iu = __fadd2_rn(x3, x4);
            const float2 rd = __fadd2_rn(x1, x2), id = fsub2(x3, x4);
            const float2 su = __ffma2_rn(ru, ru, __fmul2_rn(iu, iu));
            const float2 sd = __ffma2_rn(rd, rd, __fmul2_rn(id, id));
            const float2 mu = make_float2(sqrt_approx(su.x), sqrt_approx(su.y));
            const float2 md = make_float2(sqrt_approx(sd.x), sqrt_approx(sd.y));
            __nv_bfloat162 hu = __floats2bfloat162_rn(mu.x, mu.y);
            __nv_bfloat162 hd = __floats2bfloat162_rn(md.x, md.y);
            hv[h8][0][i] = *reinterpret_cast<uint32_t*>(&hu);
            hv[h8][1][i] = *reinterpret_cast<uint32_t*>(&hd);
            if (PS == 2) {
              const float2 fu = fsub2(mu, __bfloat1622float2(hu));
              const float2 fd = fsub2(md, __bfloat1622float2(hd));
              __nv_bfloat162 lu = __floats2bfloat162_rn(fu.x, fu.y);
              __nv_bfloat162 ld = __floats2bfloat162_rn(fd.x, fd.y);
              lv[h8][0][i] = *reinterpret_cast<uint32_t*>(&lu);
              lv[h8][1][i] = *reinterpret_cast<uint32_t*>(&ld);
            }
          }
        }
        // the pooling MMAs of the previous tile have read the staged |Z|
        if (!mbar_wait(&sfree, sph ^ 1, wait_budget)) { fail(40); ok = false; break; }
        sph ^= 1;
        tc_fence_after();
#pragma unroll
        for (int d = 0; d < 2; ++d) {
          const uint32_t zh[8] = {hv[0][d][0], hv[0][d][1], hv[0][d][2], hv[0][d][3],
                                  hv[1][d][0], hv[1][d][1], hv[1][d][2], hv[1][d][3]};
          tmem_st8(t_zw + (d * PS) * 32, zh);
          if (PS == 2) {
            const uint32_t zl[8] = {lv[0][d][0], lv[0][d][1], lv[0][d][2], lv[0][d][3],
                                    lv[1][d][0], lv[1][d][1], lv[1][d][2], lv[1][d][3]};
            tmem_st8(t_zw + (d * PS + 1) * 32, zl);
          }
        }
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sfull);
      }
      if (!ok) break;
      // the item's pooled rows: spin d = cg >> 1, frames [NT / 2 (cg & 1), +NT / 2)
      if (!mbar_wait(&dfull, dph, wait_budget)) { fail(41); break; }
      dph ^= 1;
      tc_fence_after();
      constexpr int HF = NT / 2;
      const int d = cg >> 1, f0 = HF * (cg & 1);
      float v[HF];
      {
        const uint32_t tp = t_pool + lane_off + d * NP + f0;
        if constexpr (HF == 8) {
          uint32_t hi[8];
          tmem_ld8u(tp, hi);
          if (PS == 2) {
            uint32_t lo[8];
            tmem_ld8u(tp + NT, lo);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(hi[i]) + __uint_as_float(lo[i]);
          } else {
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(hi[i]);
          }
        } else {
          float hi[16];
          tmem_ld16(tp, hi);
          if (PS == 2) {
            float lo[16];
            tmem_ld16(tp + NT, lo);
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = hi[i] + lo[i];
          } else {
            tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = hi[i];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&dfree);
      // pair row r: channel p (up) or p + n_fr (down); the phi_F rows (p = n_fr) have no down
      // channel, the zero rows before them no output
      const int r = m0 + row;
      const bool spin = r < P.n_fr * P.n1;
      const int p = spin ? r / P.n1 : P.n_fr;
      const int lam = spin ? r - p * P.n1 : r - args.pr_phi0;
      if (r < args.n_rows && (spin || r >= args.pr_phi0) && (d == 0 || spin)) {
        const int crow = (d == 0 ? (p < P.n_fr ? p : 2 * P.n_fr) : p + P.n_fr) * P.n1 + lam;
        float* out = args.P + ((size_t)b * args.n2 + a) * (size_t)P.C * P.n1 * args.nt +
                     (size_t)crow * args.nt;
        if (args.nt == NT) {
#pragma unroll
          for (int i = 0; i < HF; i += 4)
            *reinterpret_cast<float4*>(out + f0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < HF; ++i)
            if (f0 + i < args.nt) out[f0 + i] = v[i];
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// phi_F pooling along lambda of the time-pooled rows: S2[b, a, c, lo, t] =
// sum_lambda phi_F[(lo s_F - lambda) mod N_fr] P[b, a, c, lambda, t] (or P itself for Eq. 4).
// One block per (alpha, signal) walks the channels: each channel's n1 x n_t rows (contiguous
// in P) are staged in shared memory, the next channel's already in flight in registers, and
// every output adds its n1 terms in increasing lambda.
constexpr int kPoolThreads = 256;
constexpr int kPoolRowsMax = 8192;   // n1 * n_t floats staged per channel

__global__ void __launch_bounds__(kPoolThreads)
k_pool_lambda(DevPlan Pd, const float* __restrict__ P, float* __restrict__ s2) {
  __shared__ float rows[kPoolRowsMax];
  __shared__ float phi[1024];
  const int a = blockIdx.x, b = blockIdx.y;
  const int n1 = Pd.n1, nt = Pd.n_t, nfm = Pd.N_fr - 1, C = Pd.C;
  const Rate2 A = Pd.rates2[a];
  const int nout = Pd.n_lo * nt, nrow = n1 * nt;
  float* out0 = s2 + (size_t)b * Pd.s2_stride + (size_t)a * C * Pd.n_lo * nt;
  const float* in0 = P + ((size_t)b * Pd.n2 + a) * (size_t)(C * n1) * nt;
  if (A.s == 0 || !Pd.average_fr || nrow > kPoolRowsMax || Pd.N_fr > 1024) {
    for (int c = 0; c < C; ++c) {
      float* out = out0 + (size_t)c * nout;
      const float* in = in0 + (size_t)c * nrow;
      for (int i = threadIdx.x; i < nout; i += blockDim.x) {
        if (A.s == 0) { out[i] = 0.f; continue; }
        if (!Pd.average_fr) { out[i] = in[i]; continue; }
        const int lo = i / nt, t = i % nt;
        float v = 0.f;
        for (int r = 0; r < n1; ++r) v += __ldg(&Pd.phiF[(lo * Pd.s_F - r) & nfm]) * in[r * nt + t];
        out[i] = v;
      }
    }
    return;
  }
  for (int i = threadIdx.x; i < Pd.N_fr; i += blockDim.x) phi[i] = __ldg(&Pd.phiF[i]);
  constexpr int kPer = kPoolRowsMax / kPoolThreads;   // staged floats per thread
  float nxt[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = threadIdx.x + q * kPoolThreads;
    nxt[q] = i < nrow ? in0[i] : 0.f;
  }
  for (int c = 0; c < C; ++c) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int i = threadIdx.x + q * kPoolThreads;
      if (i < nrow) rows[i] = nxt[q];
    }
    __syncthreads();
    if (c + 1 < C) {
      const float* in = in0 + (size_t)(c + 1) * nrow;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int i = threadIdx.x + q * kPoolThreads;
        if (i < nrow) nxt[q] = in[i];
      }
    }
    float* out = out0 + (size_t)c * nout;
    for (int i = threadIdx.x; i < nout; i += blockDim.x) {
      const int lo = i / nt, t = i - (i / nt) * nt;
      const int base = lo * Pd.s_F;
      float v = 0.f;
#pragma unroll 4
      for (int r = 0; r < n1; ++r) v += phi[(base - r) & nfm] * rows[r * nt + t];
      out[i] = v;
    }
    __syncthreads();
  }
}

}  // namespace

// W planes: W[c * n1 + lambda][lambda'] = h_c[(lambda - lambda') mod N_fr] for lambda' < n1, else 0;
// hi = bf16(v), lo = bf16(v - hi), separately for Re and Im, and the negated Im planes.
__global__ void k_build_wplanes(DevPlan Pd, int n1_pad, __nv_bfloat16* wr_hi, __nv_bfloat16* wi_hi,
                                __nv_bfloat16* wr_lo, __nv_bfloat16* wi_lo, __nv_bfloat16* nwi_hi,
                                __nv_bfloat16* nwi_lo) {
  const int rows = Pd.C * Pd.n1;
  const long long total = (long long)rows * n1_pad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n1_pad), lp = (int)(i % n1_pad);
    const int c = r / Pd.n1, lam = r % Pd.n1;
    float2 v = make_float2(0.f, 0.f);
    if (lp < Pd.n1) v = Pd.h[(size_t)c * Pd.N_fr + ((lam - lp) & (Pd.N_fr - 1))];
    const __nv_bfloat16 hr = __float2bfloat16_rn(v.x), hi = __float2bfloat16_rn(v.y);
    wr_hi[i] = hr;
    wi_hi[i] = hi;
    const __nv_bfloat16 wl = __float2bfloat16_rn(v.y - __bfloat162float(hi));
    wr_lo[i] = __float2bfloat16_rn(v.x - __bfloat162float(hr));
    wi_lo[i] = wl;
    nwi_hi[i] = __hneg(hi);
    nwi_lo[i] = __hneg(wl);
  }
}

// FP32 W planes for the TF32 forward: Wr, Wi [C * n1][n1_pad] rounded to TF32, zero for
// lambda' >= n1.
__global__ void k_build_wplanes32(DevPlan Pd, int n1_pad, float* wr, float* wi) {
  const long long total = (long long)Pd.C * Pd.n1 * n1_pad;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n1_pad), lp = (int)(i % n1_pad);
    const int c = r / Pd.n1, lam = r % Pd.n1;
    float2 v = make_float2(0.f, 0.f);
    if (lp < Pd.n1) v = Pd.h[(size_t)c * Pd.N_fr + ((lam - lp) & (Pd.N_fr - 1))];
    wr[i] = tf32_rna(v.x);
    wi[i] = tf32_rna(v.y);
  }
}

// W planes of the spin-pair form: row r < n_fr n1 is row lambda = r mod n1 of spin-up channel
// r / n1, rows [n_fr n1, pr_phi0) are zero and row pr_phi0 + lambda is row lambda of the
// phi_F channel 2 n_fr; BF16 hi / lo of Re and Im.
__global__ void k_build_wpair(DevPlan Pd, int n1_pad, int pr_phi0, __nv_bfloat16* wr_hi,
                              __nv_bfloat16* wi_hi, __nv_bfloat16* wr_lo, __nv_bfloat16* wi_lo) {
  const long long total = (long long)(pr_phi0 + Pd.n1) * n1_pad;
  const int spin = Pd.n_fr * Pd.n1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n1_pad), lp = (int)(i % n1_pad);
    const int c = r < spin ? r / Pd.n1 : (r < pr_phi0 ? -1 : 2 * Pd.n_fr);
    const int lam = r < spin ? r % Pd.n1 : r - pr_phi0;
    float2 v = make_float2(0.f, 0.f);
    if (lp < Pd.n1 && c >= 0) v = Pd.h[(size_t)c * Pd.N_fr + ((lam - lp) & (Pd.N_fr - 1))];
    const __nv_bfloat16 hr = __float2bfloat16_rn(v.x), hi = __float2bfloat16_rn(v.y);
    wr_hi[i] = hr;
    wi_hi[i] = hi;
    wr_lo[i] = __float2bfloat16_rn(v.x - __bfloat162float(hr));
    wi_lo[i] = __float2bfloat16_rn(v.y - __bfloat162float(hi));
  }
}

// Pooling weights, t-major: w[a * NT + t][n] = s_a phi_T[(t T - n s_a) mod N] for n < L_a and
// t < n_t, zero elsewhere; stored as hi = bf16(w) and lo = bf16(w - hi).
__global__ void k_build_wt(DevPlan Pd, int NT, int Lmax, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const long long total = (long long)Pd.n2 * NT * Lmax;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i % Lmax);
    const int row = (int)(i / Lmax);
    const int a = row / NT, t = row % NT;
    const Rate2 A = Pd.rates2[a];
    float v = 0.f;
    if (A.s > 0 && n < A.L && t < Pd.n_t) v = Pd.phiT[(t * Pd.T - n * A.s) & (Pd.N - 1)] * (float)A.s;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// ----------------------------------------------------------------------------- host side
// 32-wide k-blocks of rate alpha: lambda' from lam_min rounded down to 8, in K = 16 steps
static int tc_item_kb(int n1, int lam_min) {
  const int lm8 = lam_min & ~7;
  return (((n1 - lm8 + 15) >> 4) + 1) >> 1;
}

int tc_nt(int n_t) {
  int nt = 16;
  while (nt < n_t) nt <<= 1;
  return nt;
}

// column-tile width: 128 where the 16-frame pooling leaves the shared memory for it
static int tc_bn(const jtfs_plan* p) { return tc_nt(p->n_t) == 16 ? 128 : 64; }

bool tc_supported(const jtfs_plan* p) {
  if (p->cfg.precision == JTFS_PREC_TF32 && tc_nt(p->n_t) != 16) return false;   // 16-frame form only
  return p->n2 <= 16 && tc_nt(p->n_t) <= 64 && p->cfg.precision != JTFS_PREC_FP32_SIMT;
}

namespace {
int tp_res_kb(const jtfs_plan* p);
}  // namespace

// 32-lambda' blocks of a W tile held resident in shared memory (items with more stream W)
int tc_res_kb(const jtfs_plan* p) {
  if (p->tc_pair) return tp_res_kb(p);
  return p->cfg.precision == JTFS_PREC_BF16 ? 4 : 2;
}

namespace {
constexpr size_t kSmemBudget = 225 * 1024;

struct TcShape {
  int planes, NT, BN, NH, WS;
  size_t fixed(bool res, int res_kb) const {
    return 1024 + (res ? (size_t)planes * 2 * res_kb * kBM * kBK * 2 : 0) +
           (size_t)planes * NH * kBM * 64 * 2 + (size_t)WS * planes * NH * NT * 64 * 2;
  }
  size_t stage(bool res) const {
    return (res ? 0 : (size_t)planes * 2 * kBM * kBK * 2) + (size_t)planes * 2 * NH * kBK * 64 * 2;
  }
};

TcShape tc_shape(const jtfs_plan* p) {
  TcShape s;
  s.planes = p->cfg.precision == JTFS_PREC_FP32 ? 2 : 1;
  s.NT = tc_nt(p->n_t);
  s.BN = tc_bn(p);
  s.NH = s.BN / 64;
  s.WS = 2;
  // deepest weight ring (up to 4) that still leaves two operand stages in both forms
  for (int ws = kMaxWS; ws > 2; --ws) {
    TcShape t = s;
    t.WS = ws;
    if (t.fixed(true, tc_res_kb(p)) + 2 * t.stage(true) <= kSmemBudget &&
        t.fixed(false, 0) + 2 * t.stage(false) <= kSmemBudget) {
      s.WS = ws;
      break;
    }
  }
  return s;
}

int tc_stages_for(const jtfs_plan* p, bool res) {
  const TcShape s = tc_shape(p);
  const size_t fixed = s.fixed(res, tc_res_kb(p)), stage = s.stage(res);
  if (fixed + 2 * stage > kSmemBudget) return 0;
  return (int)std::min<size_t>(8, (kSmemBudget - fixed) / stage);
}

size_t tc_smem_for(const jtfs_plan* p, bool res) {
  const TcShape s = tc_shape(p);
  return s.fixed(res, tc_res_kb(p)) + (size_t)tc_stages_for(p, res) * s.stage(res);
}

// 16-frame form (TF32 operands): resident W tile, operand stages, the weight ring, sixteen
// 1 KB |Z| staging blocks per pooling plane and the 32 KB column-group reduction buffer.
// apl: bytes of one 128 x 32 W block (8 KB BF16, 16 KB FP32 for TF32); cpl / ppl:
// contraction / pooling planes; nya: 4 KB Y atoms per part of a column tile (2 BF16, 4 FP32).
// A pooling-weight tile has two 64-sample halves.
struct Tc16Shape {
  int apl, cpl, ppl, nya, WS, nt;
  size_t fixed(bool res, int res_kb) const {
    return 1024 + (res ? (size_t)cpl * 2 * res_kb * apl : 0) + (size_t)WS * 2 * ppl * nt * 64 * 2 +
           (size_t)kEpiWarps * ppl * 1024 + 4 * 128 * 16 * 4;
  }
  size_t stage(bool res) const {
    return (res ? 0 : (size_t)cpl * 2 * apl) + (size_t)cpl * 2 * nya * 4096;
  }
};

Tc16Shape tc16_shape(const jtfs_plan* p) {
  Tc16Shape s;
  const bool tf = p->cfg.precision == JTFS_PREC_TF32;
  s.apl = tf ? kBM * kBK * 4 : kBM * kBK * 2;
  s.cpl = p->cfg.precision == JTFS_PREC_FP32 ? 2 : 1;
  s.ppl = p->split ? 2 : 1;
  s.nya = tf ? 4 : 2;
  s.WS = kMaxWS;
  s.nt = tc_nt(p->n_t);
  return s;
}

int tc16_stages_for(const jtfs_plan* p, bool res) {
  const Tc16Shape s = tc16_shape(p);
  const size_t fixed = s.fixed(res, tc_res_kb(p)), stage = s.stage(res);
  if (fixed + 2 * stage > kSmemBudget) return 0;
  return (int)std::min<size_t>(8, (kSmemBudget - fixed) / stage);
}

size_t tc16_smem_for(const jtfs_plan* p, bool res) {
  const Tc16Shape s = tc16_shape(p);
  return s.fixed(res, tc_res_kb(p)) + (size_t)tc16_stages_for(p, res) * s.stage(res);
}

// Tensor-pooling form (k_joint_fwd_tp): resident W tile, operand stages and the weight ring
// (kMaxWS slots of ppl planes of NT x 64 BF16); |Z| is staged in tensor memory.
struct TpShape {
  int cpl, ppl, nt, res_kb;
  size_t fixed(bool res) const {
    return 1024 + (res ? (size_t)cpl * 2 * res_kb * kBM * kBK * 2 : 0) +
           (size_t)kMaxWS * ppl * nt * 64 * 2;
  }
  size_t stage(bool res) const {
    return (res ? 0 : (size_t)cpl * 2 * kBM * kBK * 2) + (size_t)cpl * 2 * 4096;
  }
};

// The resident W tile holds the most 32-lambda' blocks (up to the 5 of K = 160) that leave
// room for four operand stages.
TpShape tp_shape(const jtfs_plan* p) {
  TpShape s;
  s.cpl = p->cfg.precision == JTFS_PREC_FP32 ? 2 : 1;
  s.ppl = p->split ? 2 : 1;
  s.nt = tc_nt(p->n_t);
  for (s.res_kb = 5; s.res_kb > 2; --s.res_kb)
    if (s.fixed(true) + 4 * s.stage(true) <= kSmemBudget) break;
  return s;
}

int tp_res_kb(const jtfs_plan* p) { return tp_shape(p).res_kb; }

int tp_stages_for(const jtfs_plan* p, bool res) {
  const TpShape s = tp_shape(p);
  if (s.fixed(res) + 2 * s.stage(res) > kSmemBudget) return 0;
  return (int)std::min<size_t>(8, (kSmemBudget - s.fixed(res)) / s.stage(res));
}

size_t tp_smem_for(const jtfs_plan* p, bool res) {
  const TpShape s = tp_shape(p);
  return s.fixed(res) + (size_t)tp_stages_for(p, res) * s.stage(res);
}
}  // namespace

jtfs_status build_tc_tables(jtfs_plan* p) {
  const int NT = tc_nt(p->n_t);
  const int BN = tc_bn(p);
  p->n1_pad = (p->n1 + 63) / 64 * 64;   // W plane rows hold whole 64-column boxes
  const size_t wplane = (size_t)p->C * p->n1 * p->n1_pad;
  int Lmax = BN;
  for (int a = 0; a < p->n2; ++a)
    if (p->rates2[a].s) Lmax = std::max(Lmax, (p->rates2[a].L + BN - 1) / BN * BN);
  p->tc_wt_cols = Lmax;
  // items: (alpha, m0, n_tiles); the BF16-plane forward with 16 or 32 frames runs in the
  // spin-pair form over the pair rows and 64-sample tiles
  const bool tf = p->cfg.precision == JTFS_PREC_TF32;
  p->tc_pair = NT <= 32 && !tf;
  p->pr_phi0 = (p->n_fr * p->n1 + 31) / 32 * 32;
  p->n_pr = p->pr_phi0 + p->n1;
  const int tile_n = p->tc_pair ? 64 : BN;
  struct It { int a, m0, nt; long long cost; };
  std::vector<It> its;
  const int rows = p->tc_pair ? p->n_pr : p->C * p->n1;
  for (int a = 0; a < p->n2; ++a) {
    const Rate2& A = p->rates2[a];
    if (A.s == 0) continue;
    const int ntiles = (A.L + tile_n - 1) / tile_n;
    const int kblocks = tc_item_kb(p->n1, A.lam_min);
    for (int m0 = 0; m0 < rows; m0 += kBM) its.push_back({a, m0, ntiles, (long long)ntiles * (kblocks + 2)});
  }
  // items whose W tile fits the resident form first, longest first
  const int res_kb = tc_res_kb(p);
  auto nkb = [&](const It& x) { return tc_item_kb(p->n1, p->rates2[x.a].lam_min); };
  std::stable_sort(its.begin(), its.end(), [&](const It& x, const It& y) {
    const bool rx = nkb(x) <= res_kb, ry = nkb(y) <= res_kb;
    if (rx != ry) return rx;
    return x.cost > y.cost;
  });
  p->tc_items.clear();
  p->tc_n_res = 0;
  for (auto& it : its) {
    p->tc_items.push_back(it.a); p->tc_items.push_back(it.m0); p->tc_items.push_back(it.nt); p->tc_items.push_back(0);
    if (nkb(it) <= res_kb) ++p->tc_n_res;
  }
  size_t off = 0;
  auto place = [&](size_t bytes) { size_t at = off; off += (bytes + 1023) & ~(size_t)1023; return at; };
  size_t o_w[6];
  for (int i = 0; i < 6; ++i) o_w[i] = place(wplane * 2);
  // the spin-pair planes serve the forward and backward with 16 or 32 frames
  const bool pair_planes = NT <= 32;
  size_t o_wp[4] = {0, 0, 0, 0};
  if (pair_planes)
    for (int i = 0; i < 4; ++i) o_wp[i] = place((size_t)p->n_pr * p->n1_pad * 2);
  size_t o_w32[2] = {0, 0};
  if (tf)
    for (int i = 0; i < 2; ++i) o_w32[i] = place(wplane * 4);
  const size_t wt_elems = (size_t)p->n2 * NT * Lmax;
  const size_t o_wt = place(wt_elems * 2 * 2);
  const size_t o_items = place(std::max<size_t>(16, p->tc_items.size() * 4));
  jtfs_status st;
  if ((st = cuda_check(cudaMalloc(&p->d_tc_mem, off), "tc tables")) != JTFS_OK) return st;
  char* base = (char*)p->d_tc_mem;
  for (int i = 0; i < 6; ++i) p->d_wplanes[i] = base + o_w[i];
  for (int i = 0; i < 4; ++i) p->d_wpair[i] = pair_planes ? base + o_wp[i] : nullptr;
  if (tf)
    for (int i = 0; i < 2; ++i) p->d_wplanes32[i] = base + o_w32[i];
  p->d_wtf = base + o_wt;
  p->d_tc_items = (int*)(base + o_items);
  if (!p->tc_items.empty() &&
      (st = cuda_check(cudaMemcpy(p->d_tc_items, p->tc_items.data(), p->tc_items.size() * 4, cudaMemcpyHostToDevice), "upload")) != JTFS_OK)
    return st;
  k_build_wplanes<<<1024, 256>>>(p->dp, p->n1_pad, (__nv_bfloat16*)p->d_wplanes[0],
                                 (__nv_bfloat16*)p->d_wplanes[1], (__nv_bfloat16*)p->d_wplanes[2],
                                 (__nv_bfloat16*)p->d_wplanes[3], (__nv_bfloat16*)p->d_wplanes[4],
                                 (__nv_bfloat16*)p->d_wplanes[5]);
  if (p->d_wpair[0])
    k_build_wpair<<<1024, 256>>>(p->dp, p->n1_pad, p->pr_phi0, (__nv_bfloat16*)p->d_wpair[0],
                                 (__nv_bfloat16*)p->d_wpair[1], (__nv_bfloat16*)p->d_wpair[2],
                                 (__nv_bfloat16*)p->d_wpair[3]);
  k_build_wt<<<1024, 256>>>(p->dp, NT, Lmax, (__nv_bfloat16*)p->d_wtf,
                            (__nv_bfloat16*)p->d_wtf + wt_elems);
  if (tf)
    k_build_wplanes32<<<1024, 256>>>(p->dp, p->n1_pad, (float*)p->d_wplanes32[0],
                                     (float*)p->d_wplanes32[1]);
  return cuda_check(cudaDeviceSynchronize(), "build tc tables");
}

jtfs_status launch_joint_fwd_tc(const jtfs_plan* p, int B, const void* yhi_v, const void* ylo_v,
                                float* Pbuf, float* s2, cudaStream_t st) {
  const DevPlan& d = p->dp;
  TcMaps maps;
  std::string err;
  const int passes = p->cfg.precision == JTFS_PREC_FP32 ? 3 : 1;
  const int rows = p->tc_pair ? p->n_pr : p->C * p->n1;
  const int NT = tc_nt(p->n_t);
  const int BN = tc_bn(p);
  // TF32: FP32 W planes (rows of 32 lambda' = 128 bytes) and FP32 Y planes (atoms of 32
  // samples); otherwise BF16 planes
  const bool tf = p->cfg.precision == JTFS_PREC_TF32;
  const size_t esz = tf ? 4 : 2;
  const CUtensorMapDataType dt = tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  for (int i = 0; i < 4; ++i) {
    cuuint64_t dims[2] = {(cuuint64_t)p->n1_pad, (cuuint64_t)rows};
    cuuint64_t str[1] = {(cuuint64_t)p->n1_pad * esz};
    cuuint32_t box[2] = {kBK, kBM};
    const void* src = tf ? p->d_wplanes32[i & 1] : (p->tc_pair ? p->d_wpair[i] : p->d_wplanes[i]);
    if (!make_tmap(&maps.w[i], dt, 2, src, dims, str, box, tf ? 128 : 64, &err)) {
      set_error(err);
      return JTFS_ERR_CUDA;
    }
  }
  for (int h = 0; h < 2; ++h) {
    const char* base = (const char*)(h == 0 ? yhi_v : ylo_v);
    for (int a = 0; a < 16; ++a) {
      if (a >= p->n2 || p->rates2[a].s == 0 || (passes == 1 && h == 1)) {
        maps.y[h][a] = maps.w[0];
        continue;
      }
      const Rate2& A = p->rates2[a];
      bool okm;
      if (tf) {   // transposed planes [2B][L][kt]
        cuuint64_t dims[3] = {(cuuint64_t)A.kt, (cuuint64_t)A.L, (cuuint64_t)(2 * B)};
        cuuint64_t str[2] = {(cuuint64_t)A.kt * 4, (cuuint64_t)A.L * A.kt * 4};
        cuuint32_t box[3] = {kBK, 128, 1};
        okm = make_tmap(&maps.y[h][a], dt, 3, base + (size_t)B * 2 * A.off_yt * 4, dims, str,
                        box, 128, &err);
      } else {
        cuuint64_t dims[3] = {(cuuint64_t)A.L, (cuuint64_t)A.K, (cuuint64_t)(2 * B)};
        cuuint64_t str[2] = {(cuuint64_t)A.L * esz, (cuuint64_t)A.K * A.L * esz};
        cuuint32_t box[3] = {64, kBK, 1};
        okm = make_tmap(&maps.y[h][a], dt, 3, base + (size_t)B * 2 * A.off_y * esz, dims, str,
                        box, 128, &err);
      }
      if (!okm) {
        set_error(err);
        return JTFS_ERR_CUDA;
      }
    }
  }
  const size_t wt_elems = (size_t)p->n2 * NT * p->tc_wt_cols;
  for (int h = 0; h < 2; ++h) {
    cuuint64_t dims[2] = {(cuuint64_t)p->tc_wt_cols, (cuuint64_t)p->n2 * NT};
    cuuint64_t str[1] = {(cuuint64_t)p->tc_wt_cols * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)NT};
    if (!make_tmap(&maps.wt[h], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   (const __nv_bfloat16*)p->d_wtf + (h ? wt_elems : 0), dims, str, box, 128, &err)) {
      set_error(err);
      return JTFS_ERR_CUDA;
    }
  }
  const int n_all = (int)(p->tc_items.size() / 4);
  const bool tp = p->tc_pair;                // the spin-pair form pools on the tensor cores
  const bool f16 = NT == 16 && !tp;          // the 16-frame TF32 form
  auto stages_for = [&](bool res) {
    return tp ? tp_stages_for(p, res) : (f16 ? tc16_stages_for(p, res) : tc_stages_for(p, res));
  };
  const int n_res = stages_for(true) >= 2 ? p->tc_n_res : 0;
  if (n_all > n_res && stages_for(false) < 2) {
    set_error("tensor-core forward: no shared-memory layout for this configuration");
    return JTFS_ERR_UNSUPPORTED;
  }
  TcArgs args;
  args.B = B;
  args.passes = passes;
  args.pool_split = p->split ? 1 : 0;
  args.res_kb = tc_res_kb(p);
  args.wstages = tp || f16 ? kMaxWS : tc_shape(p).WS;
  args.n_rows = rows;
  args.pr_phi0 = p->pr_phi0;
  args.nt = p->n_t;
  args.P = Pbuf;
  args.n2 = p->n2;
  args.err = p->d_err;
  args.wait_ns = p->wait_ns;
  jtfs_status rc;
  int n_sm = 148;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, p->device);
#define JTFS_LAUNCH_TC(NTV, BNV, RESV)                                                          \
  do {                                                                                          \
    if ((rc = cuda_check(cudaFuncSetAttribute(k_joint_fwd_tc<NTV, BNV, RESV>,                 \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                              (int)smem), "attr tc")) != JTFS_OK)               \
      return rc;                                                                                \
    k_joint_fwd_tc<NTV, BNV, RESV><<<grid, kThreads, smem, st>>>(maps, args, d); ++p->prof.launches; \
  } while (0)
#define JTFS_LAUNCH_TC16(RESV, TFV)                                                             \
  do {                                                                                          \
    if ((rc = cuda_check(cudaFuncSetAttribute(k_joint_fwd_tc16<RESV, TFV>,                    \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                              (int)smem), "attr tc16")) != JTFS_OK)             \
      return rc;                                                                                \
    k_joint_fwd_tc16<RESV, TFV><<<grid, kThreads, smem, st>>>(maps, args, d); ++p->prof.launches; \
  } while (0)
#define JTFS_LAUNCH_TP1(RESV, PSV, NTV)                                                         \
  do {                                                                                          \
    if ((rc = cuda_check(cudaFuncSetAttribute(k_joint_fwd_tp<RESV, PSV, NTV>,                   \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                              (int)smem), "attr tp")) != JTFS_OK)               \
      return rc;                                                                                \
    k_joint_fwd_tp<RESV, PSV, NTV><<<grid, kTpThreads, smem, st>>>(maps, args, d);              \
    ++p->prof.launches;                                                                         \
  } while (0)
#define JTFS_LAUNCH_PAIR(RESV, PSV)                                                             \
  do {                                                                                          \
    if (NT == 16) JTFS_LAUNCH_TP1(RESV, PSV, 16); else JTFS_LAUNCH_TP1(RESV, PSV, 32);          \
  } while (0)
  for (int pass = 0; pass < 2; ++pass) {
    const bool res = pass == 0;
    const int first = res ? 0 : n_res, count = res ? n_res : n_all - n_res;
    if (count <= 0) continue;
    args.items = reinterpret_cast<const int4*>(p->d_tc_items) + first;
    args.n_base = count;
    args.n_items = count * B;
    args.stages = stages_for(res);
    const size_t smem = tp ? tp_smem_for(p, res) : (f16 ? tc16_smem_for(p, res) : tc_smem_for(p, res));
    const int grid = std::min(args.n_items, n_sm);
    if (p->tc_pair) {
      if (args.pool_split) {
        if (res) JTFS_LAUNCH_PAIR(true, 2); else JTFS_LAUNCH_PAIR(false, 2);
      } else {
        if (res) JTFS_LAUNCH_PAIR(true, 1); else JTFS_LAUNCH_PAIR(false, 1);
      }
    } else if (f16) {
      // 16 frames without the spin-pair form: the TF32 operands
      if (res) JTFS_LAUNCH_TC16(true, true); else JTFS_LAUNCH_TC16(false, true);
    } else if (NT == 32) {
      if (res) JTFS_LAUNCH_TC(32, 64, true); else JTFS_LAUNCH_TC(32, 64, false);
    } else {
      if (res) JTFS_LAUNCH_TC(64, 64, true); else JTFS_LAUNCH_TC(64, 64, false);
    }
    if ((rc = cuda_check(cudaGetLastError(), "k_joint_fwd_tc")) != JTFS_OK) return rc;
  }
#undef JTFS_LAUNCH_TC
#undef JTFS_LAUNCH_TC16
#undef JTFS_LAUNCH_PAIR
#undef JTFS_LAUNCH_TP1
  k_pool_lambda<<<dim3(p->n2, B), kPoolThreads, 0, st>>>(d, Pbuf, s2);
  ++p->prof.launches;
  return cuda_check(cudaGetLastError(), "k_pool_lambda");
}

namespace {
// Diagnostic of the bounded waits: one thread initialises a barrier that expects one arrival,
// which nothing ever makes, and waits for its first phase with the contraction kernels' own
// bounded wait.  The wait gives up after `budget` ns; the thread records kWaitDiagnosticCode
// in the status word and the kernel returns (no TMEM, no copies in flight).
constexpr int kWaitDiagnosticCode = 99;
__global__ void k_wait_diagnostic(int* err, uint64_t budget) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, budget)) atomicCAS(err, 0, kWaitDiagnosticCode);
}
}  // namespace

jtfs_status launch_wait_diagnostic(const jtfs_plan* p, uint64_t budget_ns, cudaStream_t st) {
  k_wait_diagnostic<<<1, 32, 0, st>>>(p->d_err, budget_ns);
  return cuda_check(cudaGetLastError(), "k_wait_diagnostic");
}

}  // namespace jtfs

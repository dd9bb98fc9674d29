// Tensor-core (tcgen05) forward of the joint stage (Eq. 2-3): for every rate alpha, signal b
// and tile of 128 stacked channel rows r = c * n1 + lambda,
//     Z[r, n] = sum_lambda' W[r, lambda'] Y_alpha[lambda', n]      (complex, K = lambda')
// with W[c * n1 + lambda, lambda'] = h_c[(lambda - lambda') mod N_fr], then |Z| and the phi_T
// Riemann sum over n, accumulated per row across every 128-column tile of the signal:
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
// Roles (384 threads): warp 0 = TMA producer, warp 1 = MMA issuer (and TMEM owner),
// warps 4..11 = epilogue (two warps per TMEM lane quarter, each on half of the columns).
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

constexpr int kBM = 128, kBN = 128, kBK = 32;
constexpr int kThreads = 384;
constexpr int kEpiWarp0 = 4;
constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s per wait

struct TcMaps {
  CUtensorMap w[4];        // Wr_hi, Wi_hi, Wr_lo, Wi_lo : [C*n1 rows][n1_pad] bf16
  CUtensorMap y[2][16];    // [hi/lo][alpha] : [2B][K_alpha][L_alpha] bf16 (plane 2b+part)
};

struct TcArgs {
  const int4* items;       // (alpha, m0, n_tiles, 0), longest first; item it = base it / B, b = it % B
  int n_items;             // n_base * B
  int B;
  int passes;              // 1 or 3
  int n_rows;              // C * n1
  int nt;                  // frames
  const float* wt;         // per alpha: [L_alpha padded to 128][NT] pooling weights
  const long long* wt_off; // [n2]
  float* P;                // [B][n2][C*n1][nt]
  int n2;
  int* err;                // device status word (0 = ok)
};

template <int NT>
__global__ void __launch_bounds__(kThreads, 1)
k_joint_fwd_tc(const __grid_constant__ TcMaps maps, TcArgs args, DevPlan P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int planes = args.passes == 3 ? 2 : 1;          // hi (+ lo)
  const int S = args.passes == 3 ? 3 : 4;               // pipeline stages
  const uint32_t a_plane_bytes = kBM * kBK * 2;         // 8 KB
  const uint32_t b_plane_bytes = kBK * kBN * 2;         // 8 KB
  const uint32_t stage_bytes = (a_plane_bytes + b_plane_bytes) * 2 * planes;
  __shared__ uint64_t full_bar[4], empty_bar[4], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  __shared__ volatile int stop_item;
  __shared__ uint64_t mma_done;
  __shared__ float red[kBM][NT + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 8);   // one arrive per epilogue warp
    }
    mbar_init(&mma_done, 1);
    stop_item = 0;
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
      for (int i = 0; i < 4; ++i) prefetch_tmap(&maps.w[i]);
      int stage = 0;
      uint32_t phase = 0;
      int armed[4] = {-1, -1, -1, -1};   // parity of the last load issued into each stage
      for (int it = blockIdx.x; it < args.n_items && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it / args.B];
        const int a = item.x, b = it % args.B, m0 = item.y, ntiles = item.z;
        const Rate2 A = P.rates2[a];
        const int kb0 = A.lam_min / kBK, kb1 = (P.n1 + kBK - 1) / kBK;
        for (int j = 0; j < ntiles && !abort_flag; ++j) {
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&empty_bar[stage], phase ^ 1, kWaitNs)) { fail(11); break; }
            uint8_t* st = sm + stage * stage_bytes;
            mbar_arrive_expect_tx(&full_bar[stage], stage_bytes);
            armed[stage] = (int)phase;
            for (int pl = 0; pl < planes; ++pl) {
              for (int part = 0; part < 2; ++part) {
                uint8_t* dA = st + (pl * 2 + part) * a_plane_bytes;
                tma_load_2d(dA, &maps.w[pl * 2 + part], kb * kBK, m0, &full_bar[stage]);
                uint8_t* dB = st + 2 * planes * a_plane_bytes + (pl * 2 + part) * b_plane_bytes;
                const int krow = kb * kBK - A.lam_min;
                for (int h = 0; h < 2; ++h)
                  tma_load_3d(dB + h * (kBK * 128), &maps.y[pl][a], j * kBN + h * 64, krow,
                              2 * b + part, &full_bar[stage]);
              }
            }
            if (++stage == S) { stage = 0; phase ^= 1; }
          }
        }
      }
      // every load issued has landed before the CTA may exit (bounded; immediate when the
      // MMA warp consumed them)
      for (int s2 = 0; s2 < S; ++s2)
        if (armed[s2] >= 0) mbar_wait(&full_bar[s2], (uint32_t)armed[s2], kWaitNs);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id_pos = instr_desc(kBM, kBN, 1, 1, 0, 1, 0);
      const uint32_t id_neg = instr_desc(kBM, kBN, 1, 1, 0, 1, 1);
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      for (int it = blockIdx.x; it < args.n_items && !abort_flag; it += gridDim.x) {
        const int4 item = args.items[it / args.B];
        const Rate2 A = P.rates2[item.x];
        const int kb0 = A.lam_min / kBK, kb1 = (P.n1 + kBK - 1) / kBK;
        for (int j = 0; j < item.z && !abort_flag; ++j) {
          if (!mbar_wait(&tempty[acc], acc_phase ^ 1, kWaitNs)) { fail(12); break; }
          tc_fence_after();
          const uint32_t d_re = tbase + acc * 256, d_im = d_re + 128;
          bool first = true;
          for (int kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&full_bar[stage], phase, kWaitNs)) { fail(13); break; }
            tc_fence_after();
            uint8_t* st = sm + stage * stage_bytes;
            const uint32_t sa = smem_u32(st);
            const uint32_t sb = sa + (planes == 2 ? 4 : 2) * a_plane_bytes;
            for (int ks = 0; ks < kBK / 16; ++ks) {
              // plane p (0 = hi, 1 = lo), part (0 = re, 1 = im)
              auto ad = [&](int p, int part) {
                return smem_desc(sa + (p * 2 + part) * a_plane_bytes + ks * 32, 16, 512, kSw64);
              };
              auto bd = [&](int p, int part) {
                return smem_desc(sb + (p * 2 + part) * b_plane_bytes + ks * 16 * 128, kBK * 128,
                                 1024, kSw128);
              };
              // (pa, pb) plane pairs: hi*hi, then hi*lo and lo*hi for the split
              const int npair = args.passes == 3 ? 3 : 1;
              const int pa_[3] = {0, 0, 1}, pb_[3] = {0, 1, 0};
              for (int q = 0; q < npair; ++q) {
                const int pa = pa_[q], pb = pb_[q];
                const uint32_t f = first ? 0u : 1u;
                mma_f16(d_re, ad(pa, 0), bd(pb, 0), id_pos, f);   // Wr Yr
                mma_f16(d_re, ad(pa, 1), bd(pb, 1), id_neg, 1u);  // -Wi Yi
                mma_f16(d_im, ad(pa, 0), bd(pb, 1), id_pos, f);   // Wr Yi
                mma_f16(d_im, ad(pa, 1), bd(pb, 0), id_pos, 1u);  // Wi Yr
                first = false;
              }
            }
            mma_commit(&empty_bar[stage]);
            if (++stage == S) { stage = 0; phase ^= 1; }
          }
          mma_commit(&tfull[acc]);
          if (++acc == 2) { acc = 0; acc_phase ^= 1; }
        }
      }
      // all MMAs issued by this thread have completed before TMEM is released
      mma_commit(&mma_done);
      mbar_wait(&mma_done, 0, kWaitNs);
    }
  } else if (warp >= kEpiWarp0) {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - kEpiWarp0;          // 0..7
    const int quarter = warp & 3;             // TMEM lane quarter this warp may access
    const int half = ew >> 2;                 // column half
    const int row = quarter * 32 + lane;      // tile row
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int it = blockIdx.x; it < args.n_items; it += gridDim.x) {
      const int4 item = args.items[it / args.B];
      const int a = item.x, b = it % args.B, m0 = item.y;
      const float* wt = args.wt + args.wt_off[a];
      float pacc[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) pacc[t] = 0.f;
      bool ok = true;
      for (int j = 0; j < item.z; ++j) {
        if (abort_flag || !mbar_wait(&tfull[acc], acc_phase, kWaitNs)) { fail(14); ok = false; break; }
        tc_fence_after();
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const uint32_t c_re = tbase + acc * 256 + half * 64, c_im = c_re + 128;
#pragma unroll 1
        for (int c0 = 0; c0 < 64; c0 += 16) {
          float re[16], im[16];
          tmem_ld16(c_re + lane_off + c0, re);
          tmem_ld16(c_im + lane_off + c0, im);
          tmem_wait_ld();
          const float* wrow = wt + (size_t)(j * kBN + half * 64 + c0) * NT;
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const float m = sqrtf(re[i] * re[i] + im[i] * im[i]);
            const float4* w4 = reinterpret_cast<const float4*>(wrow + i * NT);
#pragma unroll
            for (int t4 = 0; t4 < NT / 4; ++t4) {
              const float4 w = __ldg(&w4[t4]);
              pacc[4 * t4 + 0] += w.x * m;
              pacc[4 * t4 + 1] += w.y * m;
              pacc[4 * t4 + 2] += w.z * m;
              pacc[4 * t4 + 3] += w.w * m;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
        if (++acc == 2) { acc = 0; acc_phase ^= 1; }
      }
      // combine the two column halves, then write this row's pooled frames; the decision to
      // stop is sampled once between the two barriers so every epilogue warp agrees on it
      asm volatile("bar.sync 1, 256;" ::: "memory");
      if (half == 1)
#pragma unroll
        for (int t = 0; t < NT; ++t) red[row][t] = pacc[t];
      if (ew == 0 && lane == 0) stop_item = abort_flag;
      asm volatile("bar.sync 1, 256;" ::: "memory");
      const bool stop = stop_item != 0;
      if (half == 0 && ok && !stop) {
        const int r = m0 + row;
        if (r < args.n_rows) {
          float* out = args.P + (((size_t)b * args.n2 + a) * args.n_rows + r) * args.nt;
          for (int t = 0; t < args.nt; ++t) out[t] = pacc[t] + red[row][t];
        }
      }
      if (stop) break;
      asm volatile("bar.sync 1, 256;" ::: "memory");   // red[] is reused by the next item
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// phi_F pooling along lambda of the time-pooled rows: S2[b, a, c, lo, t].
__global__ void k_pool_lambda(DevPlan Pd, const float* __restrict__ P, float* __restrict__ s2) {
  const int c = blockIdx.x, a = blockIdx.y, b = blockIdx.z;
  const int n1 = Pd.n1, nt = Pd.n_t, nfm = Pd.N_fr - 1;
  const Rate2 A = Pd.rates2[a];
  float* out = s2 + (((size_t)b * Pd.n2 + a) * Pd.C + c) * (size_t)Pd.n_lo * nt;
  const float* in = P + (((size_t)b * Pd.n2 + a) * (size_t)(Pd.C * n1) + (size_t)c * n1) * nt;
  for (int i = threadIdx.x; i < Pd.n_lo * nt; i += blockDim.x) {
    if (A.s == 0) { out[i] = 0.f; continue; }
    if (!Pd.average_fr) { out[i] = in[i]; continue; }
    const int lo = i / nt, t = i % nt;
    float s = 0.f;
    for (int r = 0; r < n1; ++r) s += __ldg(&Pd.phiF[(lo * Pd.s_F - r) & nfm]) * in[r * nt + t];
    out[i] = s;
  }
}

}  // namespace

// W planes: W[c * n1 + lambda][lambda'] = h_c[(lambda - lambda') mod N_fr] for lambda' < n1, else 0;
// hi = bf16(v), lo = bf16(v - hi), separately for Re and Im.
__global__ void k_build_wplanes(DevPlan Pd, int n1_pad, __nv_bfloat16* wr_hi, __nv_bfloat16* wi_hi,
                                __nv_bfloat16* wr_lo, __nv_bfloat16* wi_lo) {
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
    wr_lo[i] = __float2bfloat16_rn(v.x - __bfloat162float(hr));
    wi_lo[i] = __float2bfloat16_rn(v.y - __bfloat162float(hi));
  }
}

// Pooling weights of rate alpha: w[n][t] = s_alpha phi_T[(t T - n s_alpha) mod N] for n < L_alpha,
// t < n_t; zero in the padding.
__global__ void k_build_wt(DevPlan Pd, int a, int NT, int Lpad, float* out) {
  const Rate2 A = Pd.rates2[a];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Lpad * NT; i += gridDim.x * blockDim.x) {
    const int n = i / NT, t = i % NT;
    float v = 0.f;
    if (A.s > 0 && n < A.L && t < Pd.n_t)
      v = Pd.phiT[(t * Pd.T - n * A.s) & (Pd.N - 1)] * (float)A.s;
    out[i] = v;
  }
}

// ----------------------------------------------------------------------------- host side
int tc_nt(int n_t) {
  int nt = 16;
  while (nt < n_t) nt <<= 1;
  return nt;
}

bool tc_supported(const jtfs_plan* p) {
  return p->n2 <= 16 && tc_nt(p->n_t) <= 64 && p->cfg.precision != JTFS_PREC_FP32_SIMT &&
         p->cfg.precision != JTFS_PREC_TF32;
}

jtfs_status build_tc_tables(jtfs_plan* p) {
  const int NT = tc_nt(p->n_t);
  p->n1_pad = (p->n1 + 63) / 64 * 64;   // W plane rows hold whole 64-column boxes
  const size_t wplane = (size_t)p->C * p->n1 * p->n1_pad;
  std::vector<long long> wt_off(p->n2);
  long long wt_len = 0;
  for (int a = 0; a < p->n2; ++a) {
    wt_off[a] = wt_len;
    const int L = p->rates2[a].s ? p->rates2[a].L : 0;
    wt_len += (long long)((L + kBN - 1) / kBN * kBN) * NT;
  }
  // items: (alpha, m0, n_tiles), longest first (cost ~ n_tiles * k-blocks)
  struct It { int a, m0, nt; long long cost; };
  std::vector<It> its;
  const int rows = p->C * p->n1;
  for (int a = 0; a < p->n2; ++a) {
    const Rate2& A = p->rates2[a];
    if (A.s == 0) continue;
    const int ntiles = (A.L + kBN - 1) / kBN;
    const int kblocks = (p->n1 + kBK - 1) / kBK - A.lam_min / kBK;
    for (int m0 = 0; m0 < rows; m0 += kBM) its.push_back({a, m0, ntiles, (long long)ntiles * (kblocks + 2)});
  }
  std::stable_sort(its.begin(), its.end(), [](const It& x, const It& y) { return x.cost > y.cost; });
  p->tc_items.clear();
  for (auto& it : its) { p->tc_items.push_back(it.a); p->tc_items.push_back(it.m0); p->tc_items.push_back(it.nt); p->tc_items.push_back(0); }
  size_t off = 0;
  auto place = [&](size_t bytes) { size_t at = off; off += (bytes + 1023) & ~(size_t)1023; return at; };
  size_t o_w[4];
  for (int i = 0; i < 4; ++i) o_w[i] = place(wplane * 2);
  const size_t o_wt = place((size_t)std::max<long long>(1, wt_len) * 4);
  const size_t o_wto = place((size_t)p->n2 * 8);
  const size_t o_items = place(std::max<size_t>(16, p->tc_items.size() * 4));
  const size_t o_err = place(16);
  jtfs_status st;
  if ((st = cuda_check(cudaMalloc(&p->d_tc_mem, off), "tc tables")) != JTFS_OK) return st;
  char* base = (char*)p->d_tc_mem;
  for (int i = 0; i < 4; ++i) p->d_wplanes[i] = base + o_w[i];
  p->d_wt = (float*)(base + o_wt);
  p->d_wt_off = (long long*)(base + o_wto);
  p->d_tc_items = (int*)(base + o_items);
  p->d_err = (int*)(base + o_err);
  if ((st = cuda_check(cudaMemcpy(p->d_wt_off, wt_off.data(), p->n2 * 8, cudaMemcpyHostToDevice), "upload")) != JTFS_OK) return st;
  if (!p->tc_items.empty() &&
      (st = cuda_check(cudaMemcpy(p->d_tc_items, p->tc_items.data(), p->tc_items.size() * 4, cudaMemcpyHostToDevice), "upload")) != JTFS_OK)
    return st;
  if ((st = cuda_check(cudaMemset(p->d_err, 0, 16), "memset")) != JTFS_OK) return st;
  k_build_wplanes<<<1024, 256>>>(p->dp, p->n1_pad, (__nv_bfloat16*)p->d_wplanes[0],
                                 (__nv_bfloat16*)p->d_wplanes[1], (__nv_bfloat16*)p->d_wplanes[2],
                                 (__nv_bfloat16*)p->d_wplanes[3]);
  for (int a = 0; a < p->n2; ++a) {
    const int L = p->rates2[a].s ? p->rates2[a].L : 0;
    const int Lpad = (L + kBN - 1) / kBN * kBN;
    if (Lpad == 0) continue;
    k_build_wt<<<(Lpad * NT + 255) / 256, 256>>>(p->dp, a, NT, Lpad, p->d_wt + wt_off[a]);
  }
  return cuda_check(cudaDeviceSynchronize(), "build tc tables");
}

size_t tc_smem_bytes(const jtfs_plan* p) {
  const int passes = p->cfg.precision == JTFS_PREC_FP32 ? 3 : 1;
  const int planes = passes == 3 ? 2 : 1;
  const int S = passes == 3 ? 3 : 4;
  return 1024 + (size_t)S * (kBM * kBK * 2 + kBK * kBN * 2) * 2 * planes;
}

jtfs_status launch_joint_fwd_tc(const jtfs_plan* p, int B, const void* yhi_v, const void* ylo_v,
                                float* Pbuf, float* s2, cudaStream_t st) {
  const __nv_bfloat16* yhi = (const __nv_bfloat16*)yhi_v;
  const __nv_bfloat16* ylo = (const __nv_bfloat16*)ylo_v;
  const DevPlan& d = p->dp;
  TcMaps maps;
  std::string err;
  const int passes = p->cfg.precision == JTFS_PREC_FP32 ? 3 : 1;
  const int rows = p->C * p->n1;
  for (int i = 0; i < 4; ++i) {
    if (passes == 1 && i >= 2) { maps.w[i] = maps.w[0]; continue; }
    cuuint64_t dims[2] = {(cuuint64_t)p->n1_pad, (cuuint64_t)rows};
    cuuint64_t str[1] = {(cuuint64_t)p->n1_pad * 2};
    cuuint32_t box[2] = {kBK, kBM};
    if (!make_tmap(&maps.w[i], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p->d_wplanes[i], dims, str,
                   box, 64, &err)) {
      set_error(err);
      return JTFS_ERR_CUDA;
    }
  }
  for (int h = 0; h < 2; ++h) {
    const __nv_bfloat16* base = h == 0 ? yhi : ylo;
    for (int a = 0; a < 16; ++a) {
      if (a >= p->n2 || p->rates2[a].s == 0 || (passes == 1 && h == 1)) {
        maps.y[h][a] = maps.w[0];
        continue;
      }
      const Rate2& A = p->rates2[a];
      cuuint64_t dims[3] = {(cuuint64_t)A.L, (cuuint64_t)A.K, (cuuint64_t)(2 * B)};
      cuuint64_t str[2] = {(cuuint64_t)A.L * 2, (cuuint64_t)A.K * A.L * 2};
      cuuint32_t box[3] = {64, kBK, 1};
      if (!make_tmap(&maps.y[h][a], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                     base + (size_t)B * 2 * A.off_y, dims, str, box, 128, &err)) {
        set_error(err);
        return JTFS_ERR_CUDA;
      }
    }
  }
  TcArgs args;
  args.items = reinterpret_cast<const int4*>(p->d_tc_items);
  args.n_items = (int)(p->tc_items.size() / 4) * B;
  args.B = B;
  args.passes = passes;
  args.n_rows = rows;
  args.nt = p->n_t;
  args.wt = p->d_wt;
  (void)ylo;
  args.wt_off = p->d_wt_off;
  args.P = Pbuf;
  args.n2 = p->n2;
  args.err = p->d_err;
  const size_t smem = tc_smem_bytes(p);
  int n_sm = 148;
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, p->device);
  const int grid = std::min(args.n_items, n_sm);
  const int nt = tc_nt(p->n_t);
  jtfs_status rc;
#define JTFS_LAUNCH_TC(NTV)                                                                     \
  do {                                                                                          \
    if ((rc = cuda_check(cudaFuncSetAttribute(k_joint_fwd_tc<NTV>,                            \
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                              (int)smem), "attr tc")) != JTFS_OK)               \
      return rc;                                                                                \
    k_joint_fwd_tc<NTV><<<grid, kThreads, smem, st>>>(maps, args, d);                          \
  } while (0)
  if (nt == 16) JTFS_LAUNCH_TC(16);
  else if (nt == 32) JTFS_LAUNCH_TC(32);
  else JTFS_LAUNCH_TC(64);
#undef JTFS_LAUNCH_TC
  if ((rc = cuda_check(cudaGetLastError(), "k_joint_fwd_tc")) != JTFS_OK) return rc;
  k_pool_lambda<<<dim3(p->C, p->n2, B), 256, 0, st>>>(d, Pbuf, s2);
  return cuda_check(cudaGetLastError(), "k_pool_lambda");
}

}  // namespace jtfs

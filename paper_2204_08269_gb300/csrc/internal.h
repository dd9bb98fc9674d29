// Internal declarations of libjtfs: the plan, per-row schedule records and kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/jtfs.h"

namespace jtfs {

constexpr int kMaxLogL = 14;          // longest row FFT kept in shared memory: 2^14 complex
constexpr int kSupportSigmas = 8;     // band-pass filters are stored on xi +- 8 sigma (e^-32)
constexpr int kBandSigmas = 4;        // band edges used by the subsampling schedule

// One first-order row lambda (Sec. 2): stride, length, offsets and filter support.
struct Row1 {
  int s;        // stride s_lambda
  int L;        // N / s
  int logL;
  int off_u;    // offset of the row in a packed [u1_len] float array
  int off_uh;   // offset of the row's half spectrum (L/2 complex) in a packed array
  int ks;       // first bin of the filter support on the N grid (>= 1)
  int kl;       // number of support bins
  int off_v;    // offset of the support values in the psi1 table
};

// One second-order time rate alpha (Eq. 1, Eq. 3): stride, length and contraction rows.
struct Rate2 {
  int s;        // stride s_alpha (0 when the rate is skipped)
  int L;        // N / s
  int logL;
  int lam_min;  // first lambda' row with a non-zero Y_alpha row
  int K;        // n1 - lam_min rows of Y_alpha
  int k2e;      // end of psi-hat_alpha's support on the N grid (bins >= k2e hold < e^-32)
  int kt;       // lambda' columns of the transposed TF32 planes: from lam_min & ~7, padded to 4
  long long off_y;  // offset of Y_alpha (K x L complex) in a packed per-signal array
  long long off_yt; // offset of the transposed plane (L x kt) in a packed per-signal array
};

// Device-side constants of a plan (passed by value to kernels).
struct DevPlan {
  int N, logN, T, n_t, n1, n2, n_fr, C, N_fr, s_F, n_lo, average_fr;
  int n_phi;              // phi_t paths after the psi_t paths of S2 (0, 1, n_fr or n_fr + 1)
  int phi_psi;            // 1: the first n_fr phi_t paths are phi_T x psi_{beta,+1}
  int s2_stride;          // floats of S2 per signal: (n2 C + n_phi) n_lo n_t
  int TW, logTW;          // twiddle table length (>= every FFT length and N)
  int D, M, logM;         // decimation of the length-N FFT: N = D * M, M <= 2^kMaxLogL
  int K2max;              // width of the psi2 table (bins 0..K2max-1 on the N grid)
  long long u1_len, uh_len, y_len, yt_len;
  const Row1* rows1;      // [n1]
  const Rate2* rates2;    // [n2]
  const float* psi1;      // packed support values of psi1
  const float* psi2;      // [n2][K2max]
  const float* phiT;      // [N] time-domain lowpass phi_T[n]
  const float* phiT_lo;   // [N] phi_T[n] - phiT[n] (FP32), for the compensated S0 sums
  const float* phiThat;   // [phiT_kmax + 1] its spectrum phi-hat(q / N), q = 0..phiT_kmax (the
                          // bins phi_T is built from; beyond them phi-hat < e^-72)
  int phiT_kmax;
  const float* phiF;      // [N_fr] phi_F[m]
  const float2* h;        // [C][N_fr] log-frequency filters h_c[m]
  const float2* tw;       // [TW] exp(-2 pi i j / TW)
  const float2* twl;      // per-length tables: for L = 2^l, entries [2^(l-1) - 1, 2^l - 1) hold
                          // exp(-2 pi i m / L), m < L / 2 (contiguous reads in every stage)
  const int2* gx_lam;     // [N/2 / 256] lambda range touching each 256-bin block of x-hat
};

// Twiddles of the length-2^logL FFT (half table, exp(-2 pi i m / L) for m < L / 2).
__host__ __device__ inline const float2* twl_for(const DevPlan& P, int logL) {
  return P.twl + ((logL > 0 ? (1 << (logL - 1)) : 1) - 1);
}

}  // namespace jtfs

namespace jtfs {
// Stages timed by the optional profiler (CUDA events on the launching stream).
enum Stage {
  kStXfft = 0, kStS0, kStScalogram, kStSecondOrder, kStJointFwd, kStUhFromU1, kStJointBwd,
  kStSecondOrderBwd, kStStage1Bwd, kStGx, kNumStages
};
struct ProfRec { int stage; cudaEvent_t a, b; };
struct Profiler {
  bool on = false;
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  long long launches = 0;   // kernels launched by forward/backward calls
};
}  // namespace jtfs

struct jtfs_plan {
  jtfs_config cfg;
  int64_t N;
  int device;
  int n1, n2, n_fr, C, n_t, N_fr, s_F, n_lo;
  int n_phi = 0, phi_psi = 0;  // phi_t paths (see DevPlan)
  int s2_paths = 0;            // n2 C + n_phi
  std::vector<double> xi1, sg1, xi2, sg2, xi_fr, sg_fr;  // lambda ascending; alpha, beta descending
  double c1, c2, c_fr;
  std::vector<jtfs::Row1> rows1;
  std::vector<jtfs::Rate2> rates2;
  std::vector<int> pairs;  // (alpha, lambda') work items of the second-order kernels
  std::vector<int> rowitems;  // (alpha, lambda'_0, G, 0): G rows of one rate per CTA
  int rows_cap;               // samples one row item holds (G L_alpha <= rows_cap)
  int row_threads = 256;      // threads per CTA of the row producer (autotuned)
  bool split = false;         // BF16 hi / lo split (FP32-grade products; TF32 plans' backward)
  void* d_wplanes32[2] = {nullptr, nullptr};   // Wr, Wi FP32 [C * n1][n1_pad] (TF32 forward)
  int* d_rowitems;
  void* d_rowitems_own = nullptr;   // the autotuner's item table, when it replaced the default
  std::vector<int> items;  // (alpha, first column) work items of the joint backward
  long long u1_len, uh_len, y_len, yt_len;
  int L1max, L2max;
  jtfs::DevPlan dp;
  // device allocations
  void* d_mem;
  size_t d_bytes;
  int* d_pairs;
  int* d_items;
  // tensor-core contraction (precisions FP32 / BF16)
  bool use_tc;
  int n1_pad;                  // lambda' columns of the W planes (multiple of 32)
  void* d_wplanes[6];          // Wr_hi, Wi_hi, Wr_lo, Wi_lo, -Wi_hi, -Wi_lo: [C * n1][n1_pad] bf16
  bool tc_pair = false;        // forward in the spin-pair form (16 or 32 frames, BF16 planes)
  int pr_phi0 = 0;             // first phi_F pair row: n_fr n1 rounded up to 32 (zero rows
                               // between), so 32-row chunks never mix spin and phi_F rows
  int n_pr = 0;                // pair rows pr_phi0 + n1
  void* d_wpair[4] = {nullptr, nullptr, nullptr, nullptr};   // Wr_hi, Wi_hi, Wr_lo, Wi_lo of
                               // the spin-up and phi_F rows: [n_pr][n1_pad] bf16 (16 or 32 frames)
  void* d_wtf;                 // pooling weights hi / lo: [n2 * NT][tc_wt_cols] bf16
  int tc_wt_cols;
  std::vector<int> tc_items;   // (alpha, m0, n_tiles, 0) per signal; resident-W items first
  int tc_n_res;                // items whose W tile fits the resident form
  int* d_tc_items;
  int* d_err;                  // device status word: 0 ok, kErrNumeric after a non-finite
                               // output, any other code from a bounded wait that gave up
  uint64_t wait_ns = 2000000000ull;   // budget of every bounded device wait (ns)
  bool check_finite = false;   // scan the outputs for NaN / Inf after each call
  void* d_tc_mem;
  // tensor-core backward of the joint stage
  bool use_tcb;
  std::vector<int> tcb_items;  // (alpha, n0, lambda' start, K1) per signal; K1 <= 96 first
  int tcb_n_res;               // items with K1 <= 96
  std::vector<int> tcbf_items; // (alpha, n0, lam_min & ~7, K1): the fast backward form, the
  int tcbf_n1;                 // tcbf_n1 items with K1 <= 64 first
  int tcbf_n2a = 0;            // of the two-atom items, those with K1 <= 96 (first)
  int tcbf_n3 = 0;             // three-atom items (K1 <= 160, spin-pair form), last
  int* d_tcbf_items;
  std::vector<int> tcb_fb_items;     // (alpha, n0): rates past the tensor-core backward's
  std::vector<int> tcb_fb_rowitems;  // lambda' capacity, on CUDA cores; their Y row items
  int* d_tcb_fb_items = nullptr;
  int* d_tcb_fb_rowitems = nullptr;
  int tcb_fb_cap = 0;                // samples of the largest of those row items
  int* d_tcb_items;
  void* d_wtb;                 // [rows][NT] bf16 pooling weights (time-major)
  int* d_wtb_row0;             // [n2]
  int tcb_wt_rows;
  void* d_tcb_mem;
  mutable jtfs::Profiler prof;
};

namespace jtfs {

// status-word code of the opt-in non-finite output check (wait codes are below 100)
constexpr int kErrNumeric = 1000;

void set_error(const std::string& msg);
jtfs_status cuda_check(cudaError_t e, const char* what);

// plan construction (kernels_plan.cu)
jtfs_status build_tables(jtfs_plan* p);

// forward / backward launchers (kernels_fwd.cu, kernels_bwd.cu)
struct Workspace {
  float2* xh;      // [B][N/2]
  float2* xsub;    // [B][N]  (D sub-spectra of length M)
  float* u1;       // [B][u1_len]
  float2* uh;      // [B][uh_len]
  float2* y;       // [B][y_len]
  float2* gy;      // [B][y_len]
  float* gu1;      // [B][u1_len]
  float2* gf;      // [B][u1_len]  (per row L complex)
  float2* gxh;     // [B][N/2]
  void* ybh;       // [B * y_len * 2] bf16 (tensor-core path)
  void* ybl;       // [B * y_len * 2] bf16 (three-pass split only)
  float* yt;       // [B * yt_len * 2] FP32 transposed Y planes (TF32 contraction only)
  float* pbuf;     // [B][n2][C * n1][n_t] time-pooled rows
  void* g1;        // phi_F adjoint of g_S2 (tensor-core backward), bf16
  float* s0;       // [B][n_t]        S0, S1, S2 of the 2-D output mode (packed at the end)
  float* s1;       // [B][n1][n_t]
  float* s2;       // [B][s2_stride]
  float* gs0;      // cotangents of the 2-D output mode, unpacked
  float* gs1;
  float* gs2;
  float* s1phi;    // [B][n1][n_t] S1 rebuilt from the checkpoint (phi_t paths, backward)
  float* gs1phi;   // [B][n1][n_t] g_S1 plus the phi_t paths' adjoint
};
size_t workspace_layout(const jtfs_plan* p, int64_t B, bool with_grad, char* base, Workspace* w);

// Records an event pair around a stage when profiling is on; counts launches always.
struct StageScope {
  const jtfs_plan* p;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageScope(const jtfs_plan* p_, int stage_, cudaStream_t st_, int n_launch);
  ~StageScope();
};

// row items of the batched second-order producer for a capacity of `cap` samples per CTA
std::vector<int> build_rowitems(const jtfs_plan* p, int cap);
jtfs_status autotune_rows(jtfs_plan* p, int B, const Workspace& w, cudaStream_t st,
                          int* best_threads, int* best_cap, float* best_ms);

// tensor-core contraction (kernels_tc.cu)
bool tc_supported(const jtfs_plan* p);
int tc_nt(int n_t);
int tc_res_kb(const jtfs_plan* p);
jtfs_status build_tc_tables(jtfs_plan* p);
// phi_t paths (kernels_phi.cu): forward from S1 into the tail of each signal's S2; backward
// adds their adjoint to g_S1; S1 rebuilt from the checkpoint; the 2-D output packing.
bool phi_supported(const jtfs_plan* p);
jtfs_status launch_phi_forward(const jtfs_plan* p, int B, const float* s1, float* s2,
                               cudaStream_t st);
jtfs_status launch_s1_from_u1(const jtfs_plan* p, int B, const float* u1, float* s1,
                              cudaStream_t st);
jtfs_status launch_phi_backward(const jtfs_plan* p, int B, const float* s1, const float* gs2,
                                const float* gs1, float* gs1_out, cudaStream_t st);
jtfs_status launch_pack_2d(const jtfs_plan* p, int B, const float* s0, const float* s1,
                           const float* s2, float* out, bool unpack, cudaStream_t st);
jtfs_status launch_scat1d_forward(const jtfs_plan* p, const float* x, int B, float* s0, float* s1,
                                  float* s2t, float* u1, const Workspace& w, cudaStream_t st);
jtfs_status launch_scat1d_backward(const jtfs_plan* p, const float* x, const float* u1, int B,
                                   const float* gs0, const float* gs1, const float* gs2t,
                                   float* gx, const Workspace& w, cudaStream_t st);
jtfs_status launch_wait_diagnostic(const jtfs_plan* p, uint64_t budget_ns, cudaStream_t st);
jtfs_status launch_joint_fwd_tc(const jtfs_plan* p, int B, const void* yhi, const void* ylo,
                                float* Pbuf, float* s2, cudaStream_t st);

bool tcb_supported(const jtfs_plan* p);
jtfs_status build_tcb_tables(jtfs_plan* p);
size_t tcb_g1_bytes(const jtfs_plan* p, int64_t B);
jtfs_status launch_joint_bwd_tc(const jtfs_plan* p, int B, const void* yhi, const void* ylo,
                                const float* gs2, void* g1buf, float2* gy, cudaStream_t st);

jtfs_status launch_forward(const jtfs_plan* p, const float* x, int B, float* s0, float* s1,
                           float* s2, float* u1, const Workspace& w, cudaStream_t st);
jtfs_status launch_backward(const jtfs_plan* p, const float* x, const float* u1, int B,
                            const float* gs0, const float* gs1, const float* gs2, float* gx,
                            const Workspace& w, cudaStream_t st, bool fused = false);
// true when a fused step can hand the forward's BF16 Y planes to the backward
bool backward_reuses_forward(const jtfs_plan* p);

}  // namespace jtfs

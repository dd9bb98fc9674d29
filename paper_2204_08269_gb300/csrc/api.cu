// C ABI of libjtfs (include/jtfs.h): plan construction on the host (filterbank rule,
// subsampling schedule, table layout), argument validation and launch sequencing.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <initializer_list>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace jtfs {

thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

jtfs_status cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return JTFS_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return JTFS_ERR_CUDA;
}

namespace {

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

// Morlet bank of Sec. 2 / Eq. 1 under the repository's filterbank rule: constant-Q centre
// frequencies xi_0 2^{-k/Q} with widths rho xi (neighbours cross at half maximum) while the
// width stays >= sigma_min = 0.1 2^-J, then a linearly spaced tail of width sigma_min spaced
// one full width at half maximum apart.  Highest frequency first.
bool morlet_bank(int J, int Q, std::vector<double>& xi, std::vector<double>& sg) {
  const double fwhm = 2.0 * std::sqrt(2.0 * std::log(2.0));
  const double rho = (1.0 - std::pow(2.0, -1.0 / Q)) / fwhm;
  const double xi0 = std::min(0.35, 0.5 / (1.0 + 4.0 * rho));
  const double smin = 0.1 * std::pow(2.0, -(double)J);
  xi.clear();
  sg.clear();
  for (int k = 0; k < 100000; ++k) {
    const double x = xi0 * std::pow(2.0, -(double)k / Q);
    if (rho * x < smin) break;
    xi.push_back(x);
    sg.push_back(rho * x);
  }
  if (xi.empty()) return false;
  const double delta = fwhm * smin;
  const double xl = xi.back();
  for (int m = 1; m < 100000; ++m) {
    const double x = xl - m * delta;
    if (x < delta) break;
    xi.push_back(x);
    sg.push_back(smin);
  }
  return true;
}

int pow2_stride(double v, int o, long long cap) {
  const int e = v > 0 ? (int)std::floor(std::log2(v)) : 0;
  const long long s = 1LL << std::max(0, e - o);
  return (int)std::min(cap, s);
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

jtfs_status validate_cfg(const jtfs_config* c, int64_t N) {
  if (!c) { set_error("cfg is NULL"); return JTFS_ERR_INVALID_ARG; }
  if (!is_pow2(N) || N < 16 || N > (1LL << 20)) {
    set_error("N must be a power of two in [16, 2^20]");
    return JTFS_ERR_INVALID_ARG;
  }
  if (c->J < 1 || c->J > 24 || c->Q < 1 || c->Q > 64 || c->Q2 < 1 || c->Q2 > 64 ||
      c->J_fr < 1 || c->J_fr > 16 || c->Q_fr < 1 || c->Q_fr > 64) {
    set_error("J, Q, Q2, J_fr, Q_fr out of range");
    return JTFS_ERR_INVALID_ARG;
  }
  if (!is_pow2(c->T) || c->T > N) { set_error("T must be a power of two <= N"); return JTFS_ERR_INVALID_ARG; }
  if (c->F < 1 || c->F > (1 << 16)) { set_error("F must be in [1, 65536]"); return JTFS_ERR_INVALID_ARG; }
  if (c->average_fr != 0 && c->average_fr != 1) { set_error("average_fr must be 0 or 1"); return JTFS_ERR_INVALID_ARG; }
  if (c->oversampling < 0 || c->oversampling > 16) { set_error("oversampling must be in [0, 16]"); return JTFS_ERR_INVALID_ARG; }
  if (c->precision < 0 || c->precision > 3) { set_error("unknown precision"); return JTFS_ERR_INVALID_ARG; }
  if (c->out_3d != 0 && c->out_3d != 1) { set_error("out_3d must be 0 or 1"); return JTFS_ERR_INVALID_ARG; }
  const int br = c->branches == 0 ? (JTFS_BRANCH_PSI_PSI | JTFS_BRANCH_PSI_PHI) : c->branches;
  if ((br & ~15) || (br & 3) != 3) {
    set_error("branches must hold PSI_PSI and PSI_PHI, plus any of PHI_PSI, PHI_PHI");
    return JTFS_ERR_INVALID_ARG;
  }
  for (int i = 0; i < 3; ++i)
    if (c->reserved[i] != 0) { set_error("reserved fields must be 0"); return JTFS_ERR_INVALID_ARG; }
  return JTFS_OK;
}

}  // namespace

bool joint_simt_supported(const jtfs_plan* p);
size_t joint_fwd_smem(const jtfs_plan* p);
size_t joint_bwd_smem(const jtfs_plan* p);

static cudaEvent_t take_event(Profiler& pr) {
  if (!pr.pool.empty()) {
    cudaEvent_t e = pr.pool.back();
    pr.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

StageScope::StageScope(const jtfs_plan* p_, int stage_, cudaStream_t st_, int n_launch)
    : p(p_), stage(stage_), st(st_) {
  p->prof.launches += n_launch;
  if (p->prof.on) {
    a = take_event(p->prof);
    if (a) cudaEventRecord(a, st);
  }
}

StageScope::~StageScope() {
  if (!a) return;
  cudaEvent_t b = take_event(p->prof);
  if (!b) return;
  cudaEventRecord(b, st);
  p->prof.recs.push_back(ProfRec{stage, a, b});
}

std::vector<int> build_rowitems(const jtfs_plan* p, int cap) {
  std::vector<int> items;
  for (int a = 0; a < p->n2; ++a) {
    const Rate2& A = p->rates2[a];
    if (A.s == 0) continue;
    const int G = std::max(1, cap / A.L);
    for (int l0 = A.lam_min; l0 < p->n1; l0 += G) {
      items.push_back(a); items.push_back(l0);
      items.push_back(std::min(G, p->n1 - l0)); items.push_back(0);
    }
  }
  return items;
}

size_t workspace_layout(const jtfs_plan* p, int64_t B, bool with_grad, char* base, Workspace* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* ptr = base ? base + off : nullptr;
    off += align256(bytes);
    return ptr;
  };
  const size_t Bz = (size_t)B;
  Workspace tmp;
  Workspace& W = w ? *w : tmp;
  W.xh = (float2*)take(Bz * (p->N / 2) * 8);
  W.xsub = (float2*)take(Bz * p->N * 8);
  W.u1 = (float*)take(Bz * p->u1_len * 4);
  W.uh = (float2*)take(Bz * p->uh_len * 8);
  W.y = (float2*)take(Bz * p->y_len * 8);
  W.gy = nullptr;
  W.gu1 = nullptr;
  W.gf = nullptr;
  W.gxh = nullptr;
  W.ybh = W.ybl = nullptr;
  W.yt = nullptr;
  W.pbuf = nullptr;
  W.g1 = nullptr;
  if (p->use_tc) {
    W.ybh = take(Bz * p->y_len * 2 * 2);
    if (p->split) W.ybl = take(Bz * p->y_len * 2 * 2);
    if (p->cfg.precision == JTFS_PREC_TF32) W.yt = (float*)take(Bz * p->yt_len * 2 * 4);
    W.pbuf = (float*)take(Bz * p->n2 * (size_t)p->C * p->n1 * p->n_t * 4);
  }
  if (with_grad && p->use_tcb) W.g1 = take(tcb_g1_bytes(p, B));
  if (with_grad) {
    W.gy = (float2*)take(Bz * p->y_len * 8);
    W.gu1 = (float*)take(Bz * p->u1_len * 4);
    W.gf = (float2*)take(Bz * p->u1_len * 8);
    W.gxh = (float2*)take(Bz * (p->N / 2) * 8);
  }
  const size_t n0 = Bz * p->n_t, n1 = Bz * p->n1 * p->n_t, n2 = Bz * (size_t)p->dp.s2_stride;
  W.s0 = W.s1 = W.s2 = W.gs0 = W.gs1 = W.gs2 = W.s1phi = W.gs1phi = nullptr;
  if (!p->cfg.out_3d) {
    W.s0 = (float*)take(n0 * 4);
    W.s1 = (float*)take(n1 * 4);
    W.s2 = (float*)take(n2 * 4);
    if (with_grad) {
      W.gs0 = (float*)take(n0 * 4);
      W.gs1 = (float*)take(n1 * 4);
      W.gs2 = (float*)take(n2 * 4);
    }
  }
  if (with_grad && p->n_phi) {
    W.s1phi = (float*)take(n1 * 4);
    W.gs1phi = (float*)take(n1 * 4);
  }
  return off;
}

// Opt-in output check: any NaN or Inf among n floats records kErrNumeric in the status word.
__global__ void k_check_finite(const float* __restrict__ v, size_t n, int* err) {
  bool bad = false;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(err, 0, kErrNumeric);
}

jtfs_status check_finite(const jtfs_plan* p, cudaStream_t st,
                         std::initializer_list<std::pair<const float*, size_t>> bufs) {
  if (!p->check_finite) return JTFS_OK;
  for (const auto& b : bufs) {
    if (!b.first || b.second == 0) continue;
    const int grid = (int)std::min<size_t>(1024, (b.second + 255) / 256);
    k_check_finite<<<grid, 256, 0, st>>>(b.first, b.second, p->d_err);
    p->prof.launches += 1;
  }
  return cuda_check(cudaGetLastError(), "k_check_finite");
}

}  // namespace jtfs

using namespace jtfs;

extern "C" {

const char* jtfs_status_string(jtfs_status s) {
  switch (s) {
    case JTFS_OK: return "ok";
    case JTFS_ERR_INVALID_ARG: return "invalid argument";
    case JTFS_ERR_UNSUPPORTED: return "unsupported configuration";
    case JTFS_ERR_WORKSPACE: return "workspace too small";
    case JTFS_ERR_CUDA: return "CUDA error";
    case JTFS_ERR_TIMEOUT: return "device wait timed out";
    case JTFS_ERR_NUMERIC: return "non-finite values";
  }
  return "unknown status";
}

const char* jtfs_last_error(void) { return g_last_error.c_str(); }

void jtfs_plan_destroy(jtfs_plan* p) {
  if (!p) return;
  for (auto& r : p->prof.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : p->prof.pool) cudaEventDestroy(e);
  if (p->d_mem) cudaFree(p->d_mem);
  if (p->d_tc_mem) cudaFree(p->d_tc_mem);
  if (p->d_rowitems_own) cudaFree(p->d_rowitems_own);
  if (p->d_tcb_mem) cudaFree(p->d_tcb_mem);
  delete p;
}

jtfs_status jtfs_plan_create(const jtfs_config* cfg, int64_t N, jtfs_plan** out) {
  if (!out) { set_error("out is NULL"); return JTFS_ERR_INVALID_ARG; }
  *out = nullptr;
  jtfs_status st = validate_cfg(cfg, N);
  if (st != JTFS_OK) return st;
  jtfs_plan* p = new (std::nothrow) jtfs_plan();
  if (!p) { set_error("out of host memory"); return JTFS_ERR_INVALID_ARG; }
  p->cfg = *cfg;
  p->N = N;
  p->d_mem = nullptr;
  p->d_tc_mem = nullptr;
  p->d_tcb_mem = nullptr;
  p->d_err = nullptr;
  p->use_tc = false;
  p->use_tcb = false;
  if ((st = cuda_check(cudaGetDevice(&p->device), "cudaGetDevice")) != JTFS_OK) {
    delete p;
    return st;
  }
  auto fail = [&](jtfs_status s, const std::string& m) {
    if (!m.empty()) set_error(m);
    jtfs_plan_destroy(p);
    return s;
  };
  // --- filterbanks (lambda ascending in frequency; alpha and beta highest first) ---
  std::vector<double> xi, sg;
  if (!morlet_bank(cfg->J, cfg->Q, xi, sg)) return fail(JTFS_ERR_INVALID_ARG, "first-order bank is empty");
  p->xi1.assign(xi.rbegin(), xi.rend());
  p->sg1.assign(sg.rbegin(), sg.rend());
  if (!morlet_bank(cfg->J, cfg->Q2, p->xi2, p->sg2)) return fail(JTFS_ERR_INVALID_ARG, "second-order bank is empty");
  if (!morlet_bank(cfg->J_fr, cfg->Q_fr, p->xi_fr, p->sg_fr)) return fail(JTFS_ERR_INVALID_ARG, "frequential bank is empty");
  p->n1 = (int)p->xi1.size();
  p->n2 = (int)p->xi2.size();
  p->n_fr = (int)p->xi_fr.size();
  p->C = 2 * p->n_fr + 1;
  p->n_t = (int)(N / cfg->T);
  p->N_fr = 2 * (1 << ilog2(p->n1));
  p->s_F = 1 << (int)std::floor(std::log2((double)cfg->F));
  p->n_lo = cfg->average_fr ? (p->n1 + p->s_F - 1) / p->s_F : p->n1;
  {
    const int br = cfg->branches == 0 ? 3 : cfg->branches;
    p->phi_psi = (br & JTFS_BRANCH_PHI_PSI) != 0;
    p->n_phi = (p->phi_psi ? p->n_fr : 0) + ((br & JTFS_BRANCH_PHI_PHI) ? 1 : 0);
  }
  p->s2_paths = p->n2 * p->C + p->n_phi;
  // --- schedule (first order: envelope bandwidth 8 sigma per row) ---
  const int o = cfg->oversampling;
  p->rows1.resize(p->n1);
  long long off_u = 0, off_uh = 0, off_v = 0;
  int smin = (int)cfg->T;
  p->L1max = 0;
  for (int l = 0; l < p->n1; ++l) {
    Row1& r = p->rows1[l];
    r.s = pow2_stride(1.0 / (16.0 * p->sg1[l]), o, cfg->T);
    r.L = (int)(N / r.s);
    r.logL = ilog2(r.L);
    if (r.logL > kMaxLogL)
      return fail(JTFS_ERR_UNSUPPORTED, "a first-order row is longer than 2^14 samples (lower the oversampling)");
    r.off_u = (int)off_u;
    r.off_uh = (int)off_uh;
    off_u += r.L;
    off_uh += std::max(1, r.L / 2);
    const double lo = (p->xi1[l] - kSupportSigmas * p->sg1[l]) * (double)N;
    const double hi = (p->xi1[l] + kSupportSigmas * p->sg1[l]) * (double)N;
    r.ks = std::max(1, (int)std::ceil(lo));
    const int ke = std::min((int)(N / 2 - 1), (int)std::floor(hi));
    r.kl = std::max(0, ke - r.ks + 1);
    r.off_v = (int)off_v;
    off_v += r.kl;
    smin = std::min(smin, r.s);
    p->L1max = std::max(p->L1max, r.L);
  }
  p->u1_len = off_u;
  p->uh_len = off_uh;
  const double nyq = 0.5 / (double)smin;
  p->rates2.resize(p->n2);
  long long off_y = 0;
  p->L2max = 1;
  p->pairs.clear();
  p->items.clear();
  for (int a = 0; a < p->n2; ++a) {
    Rate2& A = p->rates2[a];
    const double lo = std::max(0.0, p->xi2[a] - kBandSigmas * p->sg2[a]);
    const double hi = std::min(p->xi2[a] + kBandSigmas * p->sg2[a], nyq);
    A.off_y = off_y;
    if (lo >= hi) {
      A.s = 0; A.L = 0; A.logL = 0; A.lam_min = p->n1; A.K = 0;
      continue;
    }
    A.s = pow2_stride(1.0 / (2.0 * (hi - lo)), o, cfg->T);
    A.L = (int)(N / A.s);
    A.logL = ilog2(A.L);
    if (A.logL > kMaxLogL)
      return fail(JTFS_ERR_UNSUPPORTED, "a second-order row is longer than 2^14 samples (lower the oversampling)");
    int lm = p->n1;
    for (int l = 0; l < p->n1; ++l)
      if (0.5 / (double)p->rows1[l].s > lo) { lm = l; break; }
    A.lam_min = lm;
    A.K = p->n1 - lm;
    off_y += (long long)A.K * A.L;
    p->L2max = std::max(p->L2max, A.L);
    for (int l = lm; l < p->n1; ++l) { p->pairs.push_back(a); p->pairs.push_back(l); }
    for (int n0 = 0; n0 < A.L; n0 += 32) { p->items.push_back(a); p->items.push_back(n0); }
  }
  p->y_len = off_y;
  if (!joint_simt_supported(p)) return fail(JTFS_ERR_UNSUPPORTED, "n1 or n1 * n_t too large for the joint-stage kernel");
  // --- device tables ---
  DevPlan& d = p->dp;
  d.N = (int)N; d.logN = ilog2(N); d.T = (int)cfg->T; d.n_t = p->n_t; d.n1 = p->n1; d.n2 = p->n2;
  d.n_fr = p->n_fr; d.C = p->C; d.N_fr = p->N_fr; d.s_F = p->s_F; d.n_lo = p->n_lo;
  d.average_fr = cfg->average_fr;
  d.n_phi = p->n_phi; d.phi_psi = p->phi_psi;
  d.s2_stride = p->s2_paths * p->n_lo * p->n_t;
  if (p->n_phi && !phi_supported(p))
    return fail(JTFS_ERR_UNSUPPORTED, "the phi_t paths need oversampling 0 and 4 n1 n_t floats of shared memory");
  d.TW = (int)N; d.logTW = d.logN;
  d.M = (int)std::min<int64_t>(N, 8192); d.logM = ilog2(d.M); d.D = (int)(N / d.M);
  d.K2max = std::max(1, p->L1max / 2);
  d.u1_len = p->u1_len; d.uh_len = p->uh_len; d.y_len = p->y_len;
  // psi-hat_alpha support end (xi + 8 sigma; both Morlet terms are below e^-32 past it) and the
  // row items of the batched second-order producer: G rows of one rate per CTA
  long long off_yt = 0;
  for (int a = 0; a < p->n2; ++a) {
    Rate2& A = p->rates2[a];
    A.k2e = (int)std::min<double>(d.K2max, std::floor((p->xi2[a] + kSupportSigmas * p->sg2[a]) * (double)N) + 1.0);
    A.kt = A.s ? (p->n1 - (A.lam_min & ~7) + 3) / 4 * 4 : 0;
    A.off_yt = off_yt;
    off_yt += (long long)A.L * A.kt;
  }
  p->yt_len = off_yt;
  d.yt_len = off_yt;
  p->rows_cap = std::max(p->L2max, 8192);
  p->rowitems = build_rowitems(p, p->rows_cap);
  // lambda range per 256-bin block of x-hat (for the gradient gather)
  const int nblk = (int)((N / 2 + 255) / 256);
  std::vector<int2> gxl(nblk);
  for (int bl = 0; bl < nblk; ++bl) {
    int lo = p->n1, hi = 0;
    const int k0 = bl * 256, k1 = k0 + 256;
    for (int l = 0; l < p->n1; ++l) {
      const Row1& r = p->rows1[l];
      if (r.kl > 0 && r.ks < k1 && r.ks + r.kl > k0) { lo = std::min(lo, l); hi = std::max(hi, l + 1); }
    }
    gxl[bl] = make_int2(lo < hi ? lo : 0, lo < hi ? hi : 0);
  }
  std::vector<float2> tw(N);
  for (long long j = 0; j < N; ++j) {
    const double ang = 2.0 * M_PI * (double)j / (double)N;
    tw[j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
  }
  // per-length half tables, L = 2^l for 1 <= l <= log2 N, packed back to back
  std::vector<float2> twl(std::max<long long>(1, N - 1));
  for (int l = 1; (1LL << l) <= N; ++l) {
    const long long L = 1LL << l, o = (L >> 1) - 1;
    for (long long m = 0; m < (L >> 1); ++m) {
      const double ang = 2.0 * M_PI * (double)m / (double)L;
      twl[o + m] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
  }
  // layout of one device allocation
  size_t off = 0;
  auto place = [&](size_t bytes) { size_t at = off; off += align256(bytes); return at; };
  const size_t o_rows = place(sizeof(Row1) * p->n1);
  const size_t o_rates = place(sizeof(Rate2) * p->n2);
  const size_t o_psi1 = place(sizeof(float) * std::max<long long>(1, off_v));
  const size_t o_psi2 = place(sizeof(float) * (size_t)p->n2 * d.K2max);
  const size_t o_phiT = place(sizeof(float) * N);
  const size_t o_phiTlo = place(sizeof(float) * N);
  // phi_T's spectrum on the bins it is built from (q <= 12 sigma_T N), FP64 then rounded
  const double sT = 0.1 / (double)p->cfg.T;
  d.phiT_kmax = std::min((int)std::ceil(12.0 * sT * N), (int)(N / 2));
  std::vector<float> phat(d.phiT_kmax + 1);
  for (int q = 0; q <= d.phiT_kmax; ++q) {
    const double w = (double)q / (double)N;
    phat[q] = (float)std::exp(-w * w / (2.0 * sT * sT));
  }
  const size_t o_phat = place(sizeof(float) * phat.size());
  const size_t o_phiF = place(sizeof(float) * p->N_fr);
  const size_t o_h = place(sizeof(float2) * (size_t)p->C * p->N_fr);
  const size_t o_tw = place(sizeof(float2) * N);
  const size_t o_twl = place(sizeof(float2) * twl.size());
  const size_t o_gx = place(sizeof(int2) * nblk);
  const size_t o_pairs = place(sizeof(int) * std::max<size_t>(2, p->pairs.size()));
  const size_t o_items = place(sizeof(int) * std::max<size_t>(2, p->items.size()));
  const size_t o_ritems = place(sizeof(int) * std::max<size_t>(4, p->rowitems.size()));
  const size_t o_err = place(16);
  p->d_bytes = off;
  if ((st = cuda_check(cudaMalloc(&p->d_mem, off), "plan tables")) != JTFS_OK) return fail(st, "");
  char* base = (char*)p->d_mem;
  d.rows1 = (const Row1*)(base + o_rows);
  d.rates2 = (const Rate2*)(base + o_rates);
  d.psi1 = (const float*)(base + o_psi1);
  d.psi2 = (const float*)(base + o_psi2);
  d.phiT = (const float*)(base + o_phiT);
  d.phiT_lo = (const float*)(base + o_phiTlo);
  d.phiThat = (const float*)(base + o_phat);
  d.phiF = (const float*)(base + o_phiF);
  d.h = (const float2*)(base + o_h);
  d.tw = (const float2*)(base + o_tw);
  d.twl = (const float2*)(base + o_twl);
  d.gx_lam = (const int2*)(base + o_gx);
  p->d_pairs = (int*)(base + o_pairs);
  p->d_items = (int*)(base + o_items);
  p->d_rowitems = (int*)(base + o_ritems);
  p->d_err = (int*)(base + o_err);
  if ((st = cuda_check(cudaMemset(p->d_err, 0, 16), "status word")) != JTFS_OK) return fail(st, "");
  struct Up { size_t at; const void* src; size_t bytes; } ups[] = {
      {o_rows, p->rows1.data(), sizeof(Row1) * p->n1},
      {o_rates, p->rates2.data(), sizeof(Rate2) * p->n2},
      {o_tw, tw.data(), sizeof(float2) * N},
      {o_phat, phat.data(), sizeof(float) * phat.size()},
      {o_twl, twl.data(), sizeof(float2) * twl.size()},
      {o_gx, gxl.data(), sizeof(int2) * nblk},
      {o_pairs, p->pairs.data(), sizeof(int) * p->pairs.size()},
      {o_items, p->items.data(), sizeof(int) * p->items.size()},
      {o_ritems, p->rowitems.data(), sizeof(int) * p->rowitems.size()},
  };
  for (const Up& u : ups)
    if (u.bytes && (st = cuda_check(cudaMemcpy(base + u.at, u.src, u.bytes, cudaMemcpyHostToDevice),
                                    "plan upload")) != JTFS_OK)
      return fail(st, "");
  if ((st = build_tables(p)) != JTFS_OK) return fail(st, "");
  p->split = cfg->precision == JTFS_PREC_FP32 || cfg->precision == JTFS_PREC_TF32;
  if (cfg->precision == JTFS_PREC_FP32 || cfg->precision == JTFS_PREC_BF16 ||
      cfg->precision == JTFS_PREC_TF32) {
    if (!tc_supported(p)) return fail(JTFS_ERR_UNSUPPORTED, "configuration outside the tensor-core kernel");
    p->use_tc = true;
    if ((st = build_tc_tables(p)) != JTFS_OK) return fail(st, "");
    if (tcb_supported(p)) {
      p->use_tcb = true;
      if ((st = build_tcb_tables(p)) != JTFS_OK) return fail(st, "");
    }
  }
  *out = p;
  return JTFS_OK;
}

jtfs_status jtfs_plan_shapes(const jtfs_plan* p, jtfs_shapes* s) {
  if (!p || !s) { set_error("NULL argument"); return JTFS_ERR_INVALID_ARG; }
  s->N = p->N; s->n1 = p->n1; s->n2 = p->n2; s->n_fr = p->n_fr; s->C = p->C; s->n_t = p->n_t;
  s->n_lam_out = p->n_lo; s->N_fr = p->N_fr; s->s_F = p->s_F;
  s->s0_len = p->n_t;
  s->s1_len = (int64_t)p->n1 * p->n_t;
  s->s2_len = (int64_t)p->s2_paths * p->n_lo * p->n_t;
  s->n_phi = p->n_phi;
  s->s2_paths = p->s2_paths;
  s->out_rows = 1 + (int64_t)p->n1 + (int64_t)p->s2_paths * p->n_lo;
  s->u1_len = p->u1_len;
  return JTFS_OK;
}

jtfs_status jtfs_plan_schedule(const jtfs_plan* p, int32_t* s1, int32_t* s2, int32_t* lam_min) {
  if (!p) { set_error("NULL plan"); return JTFS_ERR_INVALID_ARG; }
  for (int l = 0; l < p->n1 && s1; ++l) s1[l] = p->rows1[l].s;
  for (int a = 0; a < p->n2; ++a) {
    if (s2) s2[a] = p->rates2[a].s;
    if (lam_min) lam_min[a] = p->rates2[a].lam_min;
  }
  return JTFS_OK;
}

jtfs_status jtfs_workspace_bytes(const jtfs_plan* p, int64_t B, int32_t with_grad, size_t* out) {
  if (!p || !out || B < 0) { set_error("bad argument"); return JTFS_ERR_INVALID_ARG; }
  *out = workspace_layout(p, B, with_grad != 0, nullptr, nullptr);
  return JTFS_OK;
}

// Floats per signal of the three outputs as the caller sees them: S0, S1 and S2 in the 3-D
// mode; one [out_rows][n_t] block (in the s0 slot) and nothing else in the 2-D mode.
static void out_sizes(const jtfs_plan* p, size_t* n0, size_t* n1, size_t* n2) {
  if (p->cfg.out_3d) {
    *n0 = p->n_t;
    *n1 = (size_t)p->n1 * p->n_t;
    *n2 = (size_t)p->dp.s2_stride;
  } else {
    *n0 = (size_t)(1 + p->n1 + (size_t)p->s2_paths * p->n_lo) * p->n_t;
    *n1 = *n2 = 0;
  }
}

static jtfs_status check_out_args(const jtfs_plan* p, const void* a0, const void* a1,
                                  const void* a2, bool required, const char* what) {
  if (p->cfg.out_3d) {
    if (required && (!a0 || !a1 || !a2)) {
      set_error(std::string("NULL ") + what);
      return JTFS_ERR_INVALID_ARG;
    }
  } else if ((required && !a0) || a1 || a2) {
    set_error(std::string("2-D output mode: the first ") + what + " buffer holds all orders; "
              "the second and third must be NULL");
    return JTFS_ERR_INVALID_ARG;
  }
  return JTFS_OK;
}

// The forward's outputs, written where the layout wants them: the caller's buffers (3-D) or
// the workspace's, packed into the caller's single buffer afterwards (2-D).  The phi_t paths
// are computed from S1 into the tail of each signal's S2.
static jtfs_status forward_outputs(const jtfs_plan* p, const float* x, int B, float* s0,
                                   float* s1, float* s2, float* u1, const Workspace& w,
                                   cudaStream_t st, float** s1_used) {
  float* o0 = p->cfg.out_3d ? s0 : w.s0;
  float* o1 = p->cfg.out_3d ? s1 : w.s1;
  float* o2 = p->cfg.out_3d ? s2 : w.s2;
  jtfs_status rc = launch_forward(p, x, B, o0, o1, o2, u1, w, st);
  if (rc == JTFS_OK && p->n_phi) rc = launch_phi_forward(p, B, o1, o2, st);
  if (rc == JTFS_OK && !p->cfg.out_3d) rc = launch_pack_2d(p, B, o0, o1, o2, s0, false, st);
  if (s1_used) *s1_used = o1;
  return rc;
}

// The cotangents as the backward kernels take them: unpacked from the 2-D layout, and with the
// phi_t paths' adjoint added to g_S1 (their input is S1: the forward's, or rebuilt from the
// checkpoint when s1 is NULL).
static jtfs_status backward_cotangents(const jtfs_plan* p, int B, const float* x,
                                       const float* u1, const float* s1, const float** g0,
                                       const float** g1, const float** g2, const Workspace& w,
                                       cudaStream_t st) {
  (void)x;
  jtfs_status rc = JTFS_OK;
  if (!p->cfg.out_3d) {
    if (*g0) {
      rc = launch_pack_2d(p, B, w.gs0, w.gs1, w.gs2, const_cast<float*>(*g0), true, st);
      *g0 = w.gs0;
      *g1 = w.gs1;
      *g2 = w.gs2;
    } else {
      *g1 = *g2 = nullptr;
    }
  }
  if (rc == JTFS_OK && p->n_phi && *g2) {
    if (!s1) {
      rc = launch_s1_from_u1(p, B, u1, w.s1phi, st);
      s1 = w.s1phi;
    }
    if (rc == JTFS_OK) rc = launch_phi_backward(p, B, s1, *g2, *g1, w.gs1phi, st);
    *g1 = w.gs1phi;
  }
  return rc;
}

static jtfs_status check_device(const jtfs_plan* p) {
  int dev = -1;
  jtfs_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != JTFS_OK) return st;
  if (dev != p->device) { set_error("current device differs from the plan's device"); return JTFS_ERR_INVALID_ARG; }
  return JTFS_OK;
}

jtfs_status jtfs_forward(const jtfs_plan* p, const float* x, int64_t B, float* s0, float* s1,
                         float* s2, float* u1_ckpt, void* ws, size_t ws_bytes, void* stream) {
  if (!p || B < 0 || B > (1 << 20)) { set_error("bad plan or batch size"); return JTFS_ERR_INVALID_ARG; }
  if (B == 0) return JTFS_OK;
  if (!x) { set_error("NULL input"); return JTFS_ERR_INVALID_ARG; }
  jtfs_status st = check_out_args(p, s0, s1, s2, true, "output");
  if (st != JTFS_OK) return st;
  st = check_device(p);
  if (st != JTFS_OK) return st;
  const size_t need = workspace_layout(p, B, false, nullptr, nullptr);
  if (!ws || ws_bytes < need) {
    set_error("workspace needs " + std::to_string(need) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  Workspace w;
  workspace_layout(p, B, false, (char*)ws, &w);
  if ((st = forward_outputs(p, x, (int)B, s0, s1, s2, u1_ckpt ? u1_ckpt : w.u1, w,
                            (cudaStream_t)stream, nullptr)) != JTFS_OK)
    return st;
  size_t n0, n1, n2;
  out_sizes(p, &n0, &n1, &n2);
  const size_t Bz = (size_t)B;
  return check_finite(p, (cudaStream_t)stream, {{s0, Bz * n0}, {s1, Bz * n1}, {s2, Bz * n2}});
}

jtfs_status jtfs_backward(const jtfs_plan* p, const float* x, const float* u1_ckpt, int64_t B,
                          const float* g_s0, const float* g_s1, const float* g_s2, float* g_x,
                          void* ws, size_t ws_bytes, void* stream) {
  if (!p || B < 0 || B > (1 << 20)) { set_error("bad plan or batch size"); return JTFS_ERR_INVALID_ARG; }
  if (B == 0) return JTFS_OK;
  if (!x || !u1_ckpt || !g_x) { set_error("NULL x, u1_ckpt or g_x"); return JTFS_ERR_INVALID_ARG; }
  jtfs_status st = check_out_args(p, g_s0, g_s1, g_s2, false, "cotangent");
  if (st != JTFS_OK) return st;
  st = check_device(p);
  if (st != JTFS_OK) return st;
  const size_t need = workspace_layout(p, B, true, nullptr, nullptr);
  if (!ws || ws_bytes < need) {
    set_error("workspace needs " + std::to_string(need) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  Workspace w;
  workspace_layout(p, B, true, (char*)ws, &w);
  if ((st = backward_cotangents(p, (int)B, x, u1_ckpt, nullptr, &g_s0, &g_s1, &g_s2, w,
                                (cudaStream_t)stream)) != JTFS_OK)
    return st;
  if ((st = launch_backward(p, x, u1_ckpt, (int)B, g_s0, g_s1, g_s2, g_x, w,
                            (cudaStream_t)stream)) != JTFS_OK)
    return st;
  return check_finite(p, (cudaStream_t)stream, {{g_x, (size_t)B * p->N}});
}

jtfs_status jtfs_forward_backward(const jtfs_plan* p, const float* x, int64_t B,
                                  const float* g_s0, const float* g_s1, const float* g_s2,
                                  float* s0, float* s1, float* s2, float* u1_ckpt, float* g_x,
                                  void* ws, size_t ws_bytes, void* stream) {
  if (!p || B < 0 || B > (1 << 20)) { set_error("bad plan or batch size"); return JTFS_ERR_INVALID_ARG; }
  if (B == 0) return JTFS_OK;
  if (!x || !g_x) { set_error("NULL input or output"); return JTFS_ERR_INVALID_ARG; }
  jtfs_status st = check_out_args(p, s0, s1, s2, true, "output");
  if (st == JTFS_OK) st = check_out_args(p, g_s0, g_s1, g_s2, false, "cotangent");
  if (st != JTFS_OK) return st;
  st = check_device(p);
  if (st != JTFS_OK) return st;
  const size_t need = workspace_layout(p, B, true, nullptr, nullptr);
  if (!ws || ws_bytes < need) {
    set_error("workspace needs " + std::to_string(need) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  Workspace w;
  workspace_layout(p, B, true, (char*)ws, &w);
  float* u1 = u1_ckpt ? u1_ckpt : w.u1;
  cudaStream_t cs = (cudaStream_t)stream;
  float* s1_used = nullptr;
  if ((st = forward_outputs(p, x, (int)B, s0, s1, s2, u1, w, cs, &s1_used)) != JTFS_OK) return st;
  if ((st = backward_cotangents(p, (int)B, x, u1, s1_used, &g_s0, &g_s1, &g_s2, w, cs)) != JTFS_OK)
    return st;
  if ((st = launch_backward(p, x, u1, (int)B, g_s0, g_s1, g_s2, g_x, w, cs, true)) != JTFS_OK)
    return st;
  size_t n0, n1, n2;
  out_sizes(p, &n0, &n1, &n2);
  const size_t Bz = (size_t)B;
  return check_finite(p, cs, {{s0, Bz * n0}, {s1, Bz * n1}, {s2, Bz * n2}, {g_x, Bz * p->N}});
}

jtfs_status jtfs_scattering1d_forward(const jtfs_plan* p, const float* x, int64_t B, float* s0,
                                      float* s1, float* s2t, float* u1_ckpt, void* ws,
                                      size_t ws_bytes, void* stream) {
  if (!p || B < 0 || B > (1 << 20)) { set_error("bad plan or batch size"); return JTFS_ERR_INVALID_ARG; }
  if (B == 0) return JTFS_OK;
  if (!x || !s0 || !s1 || !s2t) { set_error("NULL input or output"); return JTFS_ERR_INVALID_ARG; }
  jtfs_status st = check_device(p);
  if (st != JTFS_OK) return st;
  const size_t need = workspace_layout(p, B, false, nullptr, nullptr);
  if (!ws || ws_bytes < need) {
    set_error("workspace needs " + std::to_string(need) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  Workspace w;
  workspace_layout(p, B, false, (char*)ws, &w);
  if ((st = launch_scat1d_forward(p, x, (int)B, s0, s1, s2t, u1_ckpt ? u1_ckpt : w.u1, w,
                                  (cudaStream_t)stream)) != JTFS_OK)
    return st;
  const size_t Bz = (size_t)B;
  return check_finite(p, (cudaStream_t)stream,
                      {{s0, Bz * p->n_t}, {s1, Bz * p->n1 * p->n_t},
                       {s2t, Bz * p->n2 * p->n1 * p->n_t}});
}

jtfs_status jtfs_scattering1d_backward(const jtfs_plan* p, const float* x, const float* u1_ckpt,
                                       int64_t B, const float* g_s0, const float* g_s1,
                                       const float* g_s2t, float* g_x, void* ws, size_t ws_bytes,
                                       void* stream) {
  if (!p || B < 0 || B > (1 << 20)) { set_error("bad plan or batch size"); return JTFS_ERR_INVALID_ARG; }
  if (B == 0) return JTFS_OK;
  if (!x || !u1_ckpt || !g_x) { set_error("NULL x, u1_ckpt or g_x"); return JTFS_ERR_INVALID_ARG; }
  jtfs_status st = check_device(p);
  if (st != JTFS_OK) return st;
  const size_t need = workspace_layout(p, B, true, nullptr, nullptr);
  if (!ws || ws_bytes < need) {
    set_error("workspace needs " + std::to_string(need) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  Workspace w;
  workspace_layout(p, B, true, (char*)ws, &w);
  if ((st = launch_scat1d_backward(p, x, u1_ckpt, (int)B, g_s0, g_s1, g_s2t, g_x, w,
                                   (cudaStream_t)stream)) != JTFS_OK)
    return st;
  return check_finite(p, (cudaStream_t)stream, {{g_x, (size_t)B * p->N}});
}

jtfs_status jtfs_plan_autotune(jtfs_plan* p, int64_t B, void* ws, size_t ws_bytes, void* stream,
                               int32_t* choice) {
  if (!p || B < 1 || B > (1 << 20)) { set_error("bad plan or batch size"); return JTFS_ERR_INVALID_ARG; }
  jtfs_status st = check_device(p);
  if (st != JTFS_OK) return st;
  const size_t need = workspace_layout(p, B, false, nullptr, nullptr);
  if (!ws || ws_bytes < need) {
    set_error("workspace needs " + std::to_string(need) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  Workspace w;
  workspace_layout(p, B, false, (char*)ws, &w);
  int threads = 0, cap = 0;
  float ms = 0.f;
  if ((st = autotune_rows(p, (int)B, w, (cudaStream_t)stream, &threads, &cap, &ms)) != JTFS_OK) return st;
  if (choice) {
    choice[0] = threads;
    choice[1] = cap;
    choice[2] = (int32_t)(ms * 1000.f);
  }
  return JTFS_OK;
}

jtfs_status jtfs_host_step_bytes(const jtfs_plan* p, int64_t B, size_t* out) {
  if (!p || !out || B < 0) { set_error("bad argument"); return JTFS_ERR_INVALID_ARG; }
  const size_t Bz = (size_t)B;
  size_t n0, n1, n2;
  out_sizes(p, &n0, &n1, &n2);
  size_t n = 0;
  n += align256(Bz * p->N * 4) * 2;                             // x, g_x
  n += align256(Bz * n0 * 4) * 2;                               // s0, g_s0 (or the 2-D block)
  n += align256(Bz * n1 * 4) * 2;                               // s1, g_s1
  n += align256(Bz * n2 * 4) * 2;                               // s2, g_s2
  n += align256(Bz * p->u1_len * 4);                            // checkpoint
  *out = n;
  return JTFS_OK;
}

jtfs_status jtfs_forward_backward_host(const jtfs_plan* p, const float* x_host, int64_t B,
                                       const float* g_s0_host, const float* g_s1_host,
                                       const float* g_s2_host, float* s0_host, float* s1_host,
                                       float* s2_host, float* g_x_host, void* dev_buf,
                                       size_t dev_buf_bytes, void* ws, size_t ws_bytes,
                                       void* stream) {
  if (!p || B < 0) { set_error("bad plan or batch size"); return JTFS_ERR_INVALID_ARG; }
  if (B == 0) return JTFS_OK;
  if (!x_host || !g_x_host) { set_error("NULL x or g_x"); return JTFS_ERR_INVALID_ARG; }
  size_t need = 0;
  jtfs_host_step_bytes(p, B, &need);
  if (!dev_buf || dev_buf_bytes < need) { set_error("dev_buf too small"); return JTFS_ERR_WORKSPACE; }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t Bz = (size_t)B;
  char* base = (char*)dev_buf;
  size_t off = 0;
  auto take = [&](size_t bytes) { char* q = base + off; off += align256(bytes); return q; };
  size_t n0, n1, n2;
  out_sizes(p, &n0, &n1, &n2);
  if (!p->cfg.out_3d && (s1_host || s2_host || g_s1_host || g_s2_host)) {
    set_error("2-D output mode: s0 / g_s0 hold all orders; the others must be NULL");
    return JTFS_ERR_INVALID_ARG;
  }
  const size_t bx = Bz * p->N * 4, b0 = Bz * n0 * 4, b1 = Bz * n1 * 4, b2 = Bz * n2 * 4;
  float* dx = (float*)take(bx);
  float* dgx = (float*)take(bx);
  float* ds0 = (float*)take(b0);
  float* dg0 = (float*)take(b0);
  float* ds1 = (float*)take(b1);
  float* dg1 = (float*)take(b1);
  float* ds2 = (float*)take(b2);
  float* dg2 = (float*)take(b2);
  float* du1 = (float*)take(Bz * p->u1_len * 4);
  jtfs_status rc;
  if ((rc = cuda_check(cudaMemcpyAsync(dx, x_host, bx, cudaMemcpyHostToDevice, st), "H2D x")) != JTFS_OK) return rc;
  if (g_s0_host && (rc = cuda_check(cudaMemcpyAsync(dg0, g_s0_host, b0, cudaMemcpyHostToDevice, st), "H2D g_s0")) != JTFS_OK) return rc;
  if (g_s1_host && (rc = cuda_check(cudaMemcpyAsync(dg1, g_s1_host, b1, cudaMemcpyHostToDevice, st), "H2D g_s1")) != JTFS_OK) return rc;
  if (g_s2_host && (rc = cuda_check(cudaMemcpyAsync(dg2, g_s2_host, b2, cudaMemcpyHostToDevice, st), "H2D g_s2")) != JTFS_OK) return rc;
  const bool o3 = p->cfg.out_3d != 0;
  if ((rc = jtfs_forward_backward(p, dx, B, g_s0_host ? dg0 : nullptr, g_s1_host ? dg1 : nullptr,
                                   g_s2_host ? dg2 : nullptr, ds0, o3 ? ds1 : nullptr,
                                   o3 ? ds2 : nullptr, du1, dgx, ws, ws_bytes, stream)) != JTFS_OK)
    return rc;
  if (s0_host && (rc = cuda_check(cudaMemcpyAsync(s0_host, ds0, b0, cudaMemcpyDeviceToHost, st), "D2H s0")) != JTFS_OK) return rc;
  if (s1_host && (rc = cuda_check(cudaMemcpyAsync(s1_host, ds1, b1, cudaMemcpyDeviceToHost, st), "D2H s1")) != JTFS_OK) return rc;
  if (s2_host && (rc = cuda_check(cudaMemcpyAsync(s2_host, ds2, b2, cudaMemcpyDeviceToHost, st), "D2H s2")) != JTFS_OK) return rc;
  if ((rc = cuda_check(cudaMemcpyAsync(g_x_host, dgx, bx, cudaMemcpyDeviceToHost, st), "D2H g_x")) != JTFS_OK) return rc;
  return cuda_check(cudaStreamSynchronize(st), "host step sync");
}

static const char* kStageNames[kNumStages] = {
    "x_fft", "s0", "scalogram", "second_order", "joint_fwd", "uh_from_u1", "joint_bwd",
    "second_order_bwd", "stage1_bwd", "gx"};

jtfs_status jtfs_profile_enable(const jtfs_plan* p, int32_t on) {
  if (!p) { set_error("NULL plan"); return JTFS_ERR_INVALID_ARG; }
  p->prof.on = on != 0;
  return JTFS_OK;
}

jtfs_status jtfs_profile_read(const jtfs_plan* p, double* ms, int32_t n_ms,
                              int64_t* launches) {
  if (!p || (n_ms > 0 && !ms)) { set_error("bad argument"); return JTFS_ERR_INVALID_ARG; }
  for (int i = 0; i < n_ms; ++i) ms[i] = 0.0;
  jtfs_status st = JTFS_OK;
  for (auto& r : p->prof.recs) {
    if (st == JTFS_OK) st = cuda_check(cudaEventSynchronize(r.b), "profile sync");
    float t = 0.f;
    if (st == JTFS_OK) st = cuda_check(cudaEventElapsedTime(&t, r.a, r.b), "profile elapsed");
    if (st == JTFS_OK && r.stage < n_ms) ms[r.stage] += t;
    p->prof.pool.push_back(r.a);
    p->prof.pool.push_back(r.b);
  }
  p->prof.recs.clear();
  if (launches) *launches = p->prof.launches;
  p->prof.launches = 0;
  return st;
}

const char* jtfs_profile_stage_name(int32_t i) {
  return (i >= 0 && i < kNumStages) ? kStageNames[i] : nullptr;
}

jtfs_status jtfs_sync_status(const jtfs_plan* p, void* stream) {
  if (!p) { set_error("NULL plan"); return JTFS_ERR_INVALID_ARG; }
  jtfs_status st = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "stream sync");
  if (st != JTFS_OK) return st;
  if ((st = cuda_check(cudaGetLastError(), "pending error")) != JTFS_OK) return st;
  if (p->d_err) {
    int code = 0;
    if ((st = cuda_check(cudaMemcpy(&code, p->d_err, sizeof(int), cudaMemcpyDeviceToHost), "status word")) != JTFS_OK)
      return st;
    if (code != 0) {
      if ((st = cuda_check(cudaMemset(p->d_err, 0, sizeof(int)), "clear status word")) != JTFS_OK)
        return st;
      if (code == kErrNumeric) {
        set_error("non-finite values (NaN or Inf) in the outputs of an earlier call");
        return JTFS_ERR_NUMERIC;
      }
      set_error("a bounded device wait gave up (code " + std::to_string(code) + ")");
      return JTFS_ERR_TIMEOUT;
    }
  }
  return JTFS_OK;
}

jtfs_status jtfs_plan_set_wait_budget(jtfs_plan* p, uint64_t wait_ns) {
  if (!p || wait_ns < 1000 || wait_ns > 60000000000ull) {
    set_error("wait budget must lie in [1 us, 60 s]");
    return JTFS_ERR_INVALID_ARG;
  }
  p->wait_ns = wait_ns;
  return JTFS_OK;
}

jtfs_status jtfs_plan_set_check_finite(jtfs_plan* p, int32_t on) {
  if (!p) { set_error("NULL plan"); return JTFS_ERR_INVALID_ARG; }
  p->check_finite = on != 0;
  return JTFS_OK;
}

jtfs_status jtfs_diagnose_wait_timeout(const jtfs_plan* p, uint64_t wait_ns, void* stream) {
  if (!p || wait_ns < 1000 || wait_ns > 1000000000ull) {
    set_error("diagnostic budget must lie in [1 us, 1 s]");
    return JTFS_ERR_INVALID_ARG;
  }
  jtfs_status st = check_device(p);
  if (st != JTFS_OK) return st;
  return launch_wait_diagnostic(p, wait_ns, (cudaStream_t)stream);
}

}  // extern "C"

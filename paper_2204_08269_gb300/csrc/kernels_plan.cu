// Filterbank construction on the GPU in FP64 (Sec. 2, Eq. 1): Morlet band-pass filters,
// Gaussian lowpasses, the Littlewood-Paley normalisation of each bank, and the
// time-domain log-frequency filters h_c of the joint stage.  Run once per plan; the
// kernels write FP32 tables used by every transform.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace jtfs {
namespace {

// Un-normalised analytic Morlet on 0 < w < 1/2: unit Gaussian at xi minus its DC
// correction kappa * exp(-w^2 / 2 sigma^2), kappa = exp(-xi^2 / 2 sigma^2).
__device__ double morlet64(double w, double xi, double sg) {
  if (!(w > 0.0 && w < 0.5)) return 0.0;
  const double inv = 1.0 / (2.0 * sg * sg);
  const double kappa = exp(-xi * xi * inv);
  return exp(-(w - xi) * (w - xi) * inv) - kappa * exp(-w * w * inv);
}

// Per block: min over bins j of (1 - phi(w)^2) / P(w), P = (1/2) sum_f psi_f(w)^2, w = j / G.
// Filters farther than 12 sigma from a bin (both the band and the DC term) add < e^-72 of
// a peak and are skipped; bins with P = 0 do not bound the scalar.
__global__ void k_lp_ratio(int G, int nf, const double* __restrict__ xi,
                           const double* __restrict__ sg, double sphi, double* blockmin) {
  __shared__ double red[256];
  double best = INFINITY;
  for (int j = 1 + blockIdx.x * blockDim.x + threadIdx.x; j < G / 2; j += gridDim.x * blockDim.x) {
    const double w = (double)j / (double)G;
    double P = 0.0;
    for (int f = 0; f < nf; ++f) {
      const double x = xi[f], s = sg[f];
      if (fabs(w - x) > 12.0 * s && w > 12.0 * s) continue;
      const double v = morlet64(w, x, s);
      P += v * v;
    }
    P *= 0.5;
    if (P > 0.0) {
      const double ph = exp(-w * w / (2.0 * sphi * sphi));
      best = fmin(best, (1.0 - ph * ph) / P);
    }
  }
  red[threadIdx.x] = best;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) blockmin[blockIdx.x] = red[0];
}

// psi1 support values: for row lambda, bins ks..ks+kl-1 of the N grid.
__global__ void k_fill_psi1(int N, int n1, const Row1* __restrict__ rows, const double* __restrict__ xi,
                            const double* __restrict__ sg, double c, float* out) {
  const int lam = blockIdx.y;
  if (lam >= n1) return;
  const Row1 r = rows[lam];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < r.kl; i += gridDim.x * blockDim.x) {
    const int k = r.ks + i;
    out[r.off_v + i] = (float)(c * morlet64((double)k / (double)N, xi[lam], sg[lam]));
  }
}

// psi2 dense table [n2][K2max] on the N grid (bins below the finest first-order Nyquist).
__global__ void k_fill_psi2(int N, int n2, int K2max, const double* __restrict__ xi,
                            const double* __restrict__ sg, double c, float* out) {
  const int a = blockIdx.y;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K2max; k += gridDim.x * blockDim.x)
    out[(size_t)a * K2max + k] = (float)(c * morlet64((double)k / (double)N, xi[a], sg[a]));
}

// phi_T[n] = (1/N) sum_k phi-hat(k/N) exp(2 pi i k n / N): real and even; bins beyond
// 12 sigma_T add < e^-72.  out receives the FP32 rounding of the FP64 value and out_lo the
// FP32 rounding of the remainder (phi_T = out + out_lo to about 2^-48 relative).
__global__ void k_fill_phiT(int N, int kmax, double sphi, float* out, float* out_lo) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    double acc = 1.0;
    for (int k = 1; k <= kmax; ++k) {
      const double w = (double)k / (double)N;
      const double g = exp(-w * w / (2.0 * sphi * sphi));
      const long long kn = ((long long)k * n) % N;
      const double cs = cospi(2.0 * (double)kn / (double)N);
      acc += (k == N / 2 ? 1.0 : 2.0) * g * cs;
    }
    const double v = acc / (double)N;
    const float hi = (float)v;
    out[n] = hi;
    out_lo[n] = (float)(v - (double)hi);
  }
}

// Log-frequency filters on the N_fr grid: h_c[m] = (1/N_fr) sum_j H_c(w_j) exp(2 pi i j m / N_fr),
// H_c = c_fr psi(w) (theta = +1, c < n_fr), c_fr psi(-w) (theta = -1), phi_F(w) (c = 2 n_fr).
__global__ void k_fill_fr(int Nfr, int nfr, const double* __restrict__ xi,
                          const double* __restrict__ sg, double c, double sphi, float2* h,
                          float* phiF) {
  const int ch = blockIdx.y;
  const int C = 2 * nfr + 1;
  if (ch >= C) return;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < Nfr; m += gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < Nfr; ++j) {
      const double w = (j <= Nfr / 2 ? (double)j : (double)(j - Nfr)) / (double)Nfr;
      double H;
      if (ch < nfr) H = c * morlet64(w, xi[ch], sg[ch]);
      else if (ch < 2 * nfr) H = c * morlet64(-w, xi[ch - nfr], sg[ch - nfr]);
      else H = exp(-w * w / (2.0 * sphi * sphi));
      if (H == 0.0) continue;
      const long long jm = ((long long)j * m) % Nfr;
      double sn, cs;
      sincospi(2.0 * (double)jm / (double)Nfr, &sn, &cs);
      re += H * cs;
      im += H * sn;
    }
    h[(size_t)ch * Nfr + m] = make_float2((float)(re / Nfr), (float)(im / Nfr));
    if (ch == 2 * nfr) phiF[m] = (float)(re / Nfr);
  }
}

jtfs_status lp_scalar(const std::vector<double>& xi, const std::vector<double>& sg, double sphi,
                     int G, double* scratch, double* c_out) {
  const int nf = (int)xi.size();
  double* d_xi = scratch;
  double* d_sg = scratch + nf;
  double* d_min = scratch + 2 * nf;
  const int blocks = 256;
  jtfs_status st;
  if ((st = cuda_check(cudaMemcpy(d_xi, xi.data(), nf * sizeof(double), cudaMemcpyHostToDevice),
                       "copy bank")) != JTFS_OK)
    return st;
  if ((st = cuda_check(cudaMemcpy(d_sg, sg.data(), nf * sizeof(double), cudaMemcpyHostToDevice),
                       "copy bank")) != JTFS_OK)
    return st;
  k_lp_ratio<<<blocks, 256>>>(G, nf, d_xi, d_sg, sphi, d_min);
  if ((st = cuda_check(cudaGetLastError(), "k_lp_ratio")) != JTFS_OK) return st;
  std::vector<double> mins(blocks);
  if ((st = cuda_check(cudaMemcpy(mins.data(), d_min, blocks * sizeof(double),
                                  cudaMemcpyDeviceToHost), "lp min")) != JTFS_OK)
    return st;
  double m = INFINITY;
  for (double v : mins) m = std::min(m, v);
  if (!(m > 0.0) || !std::isfinite(m)) {
    set_error("Littlewood-Paley normalisation found no bin covered by the bank");
    return JTFS_ERR_INVALID_ARG;
  }
  *c_out = std::sqrt(m);
  return JTFS_OK;
}

}  // namespace

// Fills every device table of the plan.  p->d_mem already holds the host-computed tables
// (rows, rates, twiddles, lambda ranges); this computes the LP scalars and the filters.
jtfs_status build_tables(jtfs_plan* p) {
  jtfs_status st;
  const int N = (int)p->N;
  size_t nmax = std::max({p->xi1.size(), p->xi2.size(), p->xi_fr.size()});
  double* scratch = nullptr;
  if ((st = cuda_check(cudaMalloc(&scratch, (2 * nmax + 256) * sizeof(double)), "plan scratch")) !=
      JTFS_OK)
    return st;
  const double sT = 0.1 / (double)p->cfg.T;
  const double sF = 0.1 / (double)p->cfg.F;
  st = lp_scalar(p->xi1, p->sg1, sT, N, scratch, &p->c1);
  if (st == JTFS_OK) st = lp_scalar(p->xi2, p->sg2, sT, N, scratch, &p->c2);
  if (st == JTFS_OK) st = lp_scalar(p->xi_fr, p->sg_fr, sF, p->N_fr, scratch, &p->c_fr);
  if (st != JTFS_OK) {
    cudaFree(scratch);
    return st;
  }
  // first order
  std::vector<double> buf(2 * nmax);
  auto upload = [&](const std::vector<double>& a, const std::vector<double>& b) {
    std::copy(a.begin(), a.end(), buf.begin());
    std::copy(b.begin(), b.end(), buf.begin() + a.size());
    return cuda_check(cudaMemcpy(scratch, buf.data(), 2 * a.size() * sizeof(double),
                                 cudaMemcpyHostToDevice), "copy bank");
  };
  const DevPlan& d = p->dp;
  if ((st = upload(p->xi1, p->sg1)) != JTFS_OK) goto done;
  {
    int maxkl = 0;
    for (auto& r : p->rows1) maxkl = std::max(maxkl, r.kl);
    dim3 g((maxkl + 255) / 256, p->n1);
    k_fill_psi1<<<g, 256>>>(N, p->n1, d.rows1, scratch, scratch + p->n1, p->c1,
                            const_cast<float*>(d.psi1));
  }
  if ((st = cuda_check(cudaDeviceSynchronize(), "k_fill_psi1")) != JTFS_OK) goto done;
  if ((st = upload(p->xi2, p->sg2)) != JTFS_OK) goto done;
  {
    dim3 g((d.K2max + 255) / 256, p->n2);
    k_fill_psi2<<<g, 256>>>(N, p->n2, d.K2max, scratch, scratch + p->n2, p->c2,
                            const_cast<float*>(d.psi2));
  }
  if ((st = cuda_check(cudaDeviceSynchronize(), "k_fill_psi2")) != JTFS_OK) goto done;
  {
    int kmax = (int)std::ceil(12.0 * sT * N);
    kmax = std::min(kmax, N / 2);
    k_fill_phiT<<<(N + 255) / 256, 256>>>(N, kmax, sT, const_cast<float*>(d.phiT),
                                          const_cast<float*>(d.phiT_lo));
  }
  if ((st = cuda_check(cudaDeviceSynchronize(), "k_fill_phiT")) != JTFS_OK) goto done;
  if ((st = upload(p->xi_fr, p->sg_fr)) != JTFS_OK) goto done;
  {
    dim3 g((p->N_fr + 127) / 128, p->C);
    k_fill_fr<<<g, 128>>>(p->N_fr, p->n_fr, scratch, scratch + p->n_fr, p->c_fr, sF,
                          const_cast<float2*>(d.h), const_cast<float*>(d.phiF));
  }
  st = cuda_check(cudaDeviceSynchronize(), "k_fill_fr");
done:
  cudaFree(scratch);
  return st;
}

}  // namespace jtfs

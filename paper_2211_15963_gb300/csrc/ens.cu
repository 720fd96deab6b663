// HMDA ensemble: M networks that share one graph, stepped together by one
// engine, and the FP64 diffusion ensemble Kalman analysis of Supplementary
// Algorithm 3 on the device.
//
// State of member m, region r (block of 7):
//   [theta_AMPA, theta_GABA_A, s, f, v, q, y]
// theta are natural-log scales of the region's AMPA and GABA_A maximal
// conductances (the hyperparameters; for a scale family the cdf^-1 map of
// Supplementary Sec. 6 is a plain rescale).  s, f, v, q is the
// Balloon-Windkessel state and y its output at the latest bin.
//
// Analysis (observer l sees region l's BOLD; L = R):
//   mu = mean_m X_m,  A = X - mu                          (Alg. 3 step 4)
//   c_l = A^T A[:, h_l] / (M - 1),  S_l = c_l[h_l] + G,  K_l = c_l / S_l   (step 5)
//   nu[m][l] = y_l - sqrt(G) eps[m][l] - X[m][h_l]        (step 6)
//   X'[m][c] = X[m][c] + gamma K_b[c] nu[m][b]
//              + (1 - gamma)/(L - 1) sum_{k != b} K_k[c] nu[m][k],  b = block of c
// which is step 7's fusion written out (each observer's corrected state is
// X + K_l nu_l, and component c keeps the Upsilon-weighted average of the
// observers with its own block's observer weighted by gamma).  In the global
// mode one observer sees all R signals: S = H C H^T + G I is factorised by
// Cholesky and X' = X + C H^T S^-1 (y - sqrt(G) eps - H X).
// Then theta is clipped to its prior support, f, v, q are floored, theta
// takes a random-walk step, and the members' conductances are rescaled.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "dbnet.h"
#include "engine.h"
#include "host.h"

namespace dbn {
namespace {

constexpr int kB = 7;   // values per region block
constexpr int kY = 6;   // position of y in a block

__global__ void k_gather(double* X, const double* theta, const double* bw, const double* ylast,
                         int M, int R) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * R) return;
  const int m = i / R, r = i % R;
  double* x = X + (size_t)m * kB * R + kB * r;
  x[0] = theta[2 * i];
  x[1] = theta[2 * i + 1];
  for (int k = 0; k < 4; ++k) x[2 + k] = bw[4 * i + k];
  x[6] = ylast[i];
}

// column means and deviations
__global__ void k_mean_dev(const double* X, double* mu, double* A, int M, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double s = 0.0;
  for (int m = 0; m < M; ++m) s += X[(size_t)m * n + c];
  const double mc = s / M;
  mu[c] = mc;
  for (int m = 0; m < M; ++m) A[(size_t)m * n + c] = X[(size_t)m * n + c] - mc;
}

// diffusion gains: K[l][c] = (A^T A)[c][h_l] / (M-1) / S_l
__global__ void k_gain_diffusion(const double* A, double* K, int M, int n, int L, double G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L * n) return;
  const int l = i / n, c = i % n;
  const int h = kB * l + kY;
  double cc = 0.0, ch = 0.0;
  for (int m = 0; m < M; ++m) {
    const double ah = A[(size_t)m * n + h];
    cc += A[(size_t)m * n + c] * ah;
    ch += ah * ah;
  }
  cc /= (M - 1);
  ch /= (M - 1);
  K[i] = cc / (ch + G);
}

__global__ void k_innovation(double* nu, const double* X, const double* y_obs, const double* eps,
                             int M, int R, double sd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * R) return;
  const int m = i / R, l = i % R;
  nu[i] = y_obs[l] - sd * eps[i] - X[(size_t)m * kB * R + kB * l + kY];
}

__global__ void k_fuse(double* X, const double* K, const double* nu, int M, int R, double gamma) {
  const int n = kB * R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * n) return;
  const int m = i / n, c = i % n, b = c / kB;
  const double* nm = nu + (size_t)m * R;
  double own = K[(size_t)b * n + c] * nm[b];
  double upd;
  if (R == 1) {
    upd = own;
  } else {
    double others = 0.0;
    for (int k = 0; k < R; ++k)
      if (k != b) others += K[(size_t)k * n + c] * nm[k];
    upd = gamma * own + (1.0 - gamma) / (R - 1) * others;
  }
  X[i] += upd;
}

// global mode: S[i][j] = C[h_i][h_j] + G delta_ij, and P[i][c] = C[h_i][c]
__global__ void k_cov_obs(const double* A, double* S, double* P, int M, int R, double G) {
  const int n = kB * R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < R * R) {
    const int a = i / R, b = i % R;
    const int ha = kB * a + kY, hb = kB * b + kY;
    double s = 0.0;
    for (int m = 0; m < M; ++m) s += A[(size_t)m * n + ha] * A[(size_t)m * n + hb];
    S[i] = s / (M - 1) + (a == b ? G : 0.0);
  }
  if (i < R * n) {
    const int a = i / n, c = i % n;
    const int ha = kB * a + kY;
    double s = 0.0;
    for (int m = 0; m < M; ++m) s += A[(size_t)m * n + ha] * A[(size_t)m * n + c];
    P[i] = s / (M - 1);
  }
}

// In-place Cholesky S = L L^T (lower triangle) by one block; sets *bad if S
// is not positive definite.
__global__ void k_cholesky(double* S, int R, int* bad) {
  for (int k = 0; k < R; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const double d = S[k * R + k];
      if (!(d > 0.0)) *bad = 1;
      S[k * R + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double dk = S[k * R + k];
    for (int i = k + 1 + threadIdx.x; i < R; i += blockDim.x) S[i * R + k] /= dk;
    __syncthreads();
    for (int t = threadIdx.x; t < (R - k - 1) * (R - k - 1); t += blockDim.x) {
      const int i = k + 1 + t / (R - k - 1), j = k + 1 + t % (R - k - 1);
      if (j <= i) S[i * R + j] -= S[i * R + k] * S[j * R + k];
    }
  }
}

// Solve S Z = P column by column (Z = S^-1 P, [R][n]) with the factor L.
__global__ void k_chol_solve(const double* Lf, double* P, int R, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < R; ++i) {  // L y = p
    double s = P[(size_t)i * n + c];
    for (int k = 0; k < i; ++k) s -= Lf[i * R + k] * P[(size_t)k * n + c];
    P[(size_t)i * n + c] = s / Lf[i * R + i];
  }
  for (int i = R - 1; i >= 0; --i) {  // L^T z = y
    double s = P[(size_t)i * n + c];
    for (int k = i + 1; k < R; ++k) s -= Lf[k * R + i] * P[(size_t)k * n + c];
    P[(size_t)i * n + c] = s / Lf[i * R + i];
  }
}

// X[m][c] += sum_i Z[i][c] nu[m][i]   (K = Z^T)
__global__ void k_apply_global(double* X, const double* Z, const double* nu, int M, int R) {
  const int n = kB * R;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * n) return;
  const int m = i / n, c = i % n;
  double s = 0.0;
  for (int k = 0; k < R; ++k) s += Z[(size_t)k * n + c] * nu[(size_t)m * R + k];
  X[i] += s;
}

// Sets bit 2 of *bad when the analysed ensemble holds a non-finite value
// (for instance a forecast whose hemodynamic state overflowed).
__global__ void k_check_finite(const double* X, int64_t n, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(X[i])) {
      atomicOr(bad, 2);
      return;
    }
}

// The two kernels that write the members' state do nothing when the
// analysis failed (*bad != 0), so a failed call leaves theta, the
// hemodynamic state and the region constants as they were.
__global__ void k_constrain_writeback(const double* X, double* theta, double* bw, int M, int R,
                                      double lo, double hi, double floor_, const int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * R || *bad) return;
  const int m = i / R, r = i % R;
  const double* x = X + (size_t)m * kB * R + kB * r;
  theta[2 * i] = fmin(fmax(x[0], lo), hi);
  theta[2 * i + 1] = fmin(fmax(x[1], lo), hi);
  bw[4 * i] = x[2];
  for (int k = 1; k < 4; ++k) bw[4 * i + k] = fmax(x[2 + k], floor_);
}

// Philox4x64-10 (Salmon et al., SC'11) for the analysis noise.
__device__ void philox4x64(unsigned long long c[4], unsigned long long k0, unsigned long long k1) {
  for (int r = 0; r < 10; ++r) {
    const unsigned long long m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    unsigned long long hi0 = __umul64hi(m0, c[0]), lo0 = m0 * c[0];
    unsigned long long hi1 = __umul64hi(m1, c[2]), lo1 = m1 * c[2];
    unsigned long long n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}

// Standard normals by the Box-Muller transform of two 53-bit uniforms from
// Philox counter (analysis index, i, stream, 0): out[i] for i < n.
__global__ void k_normals(double* out, int n, unsigned long long seed, unsigned long long key1,
                          unsigned long long idx, unsigned long long stream) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long c[4] = {idx, (unsigned long long)i, stream, 0ull};
  philox4x64(c, seed, key1);
  const double u1 = ((c[0] >> 11) + 1) * (1.0 / 9007199254740992.0);  // (0, 1]
  const double u2 = (c[1] >> 11) * (1.0 / 9007199254740992.0);
  out[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// theta <- clip(theta + rw_sigma xi) and the members' scaled targets:
// value = base exp(theta) for each slot's target (a conductance or I_ext).
__device__ __forceinline__ void set_target(RegionConst& rc, int target, float v) {
  if (target == DBENS_T_IEXT) rc.Iext = v;
  else if (target >= DBENS_T_AMPA && target <= DBENS_T_GABA_B) rc.g[target - DBENS_T_AMPA] = v;
}

__global__ void k_walk_rescale(double* theta, const double* xi, const double* base_g,
                               const InstDesc* insts, int M, int R, double rw, double lo,
                               double hi, int t0, int t1, const int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * R || *bad) return;
  const int m = i / R, r = i % R;
  const double ta = fmin(fmax(theta[2 * i] + rw * xi[2 * i], lo), hi);
  const double tg = fmin(fmax(theta[2 * i + 1] + rw * xi[2 * i + 1], lo), hi);
  theta[2 * i] = ta;
  theta[2 * i + 1] = tg;
  RegionConst* rc = const_cast<RegionConst*>(insts[m].rc);
  set_target(rc[r], t0, (float)(base_g[2 * r] * exp(ta)));
  set_target(rc[r], t1, (float)(base_g[2 * r + 1] * exp(tg)));
}

inline int blocks(int64_t n, int t = 128) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace
}  // namespace dbn

using namespace dbn;

struct dbens {
  std::unique_ptr<Engine> eng;
  int M = 0, R = 0;
  dbens_enkf_t enkf{};
  int target[2] = {DBENS_T_AMPA, DBENS_T_GABA_A};  // resolved DBENS_T_* of the two slots
  uint64_t seed = 0, net_id0 = 0;
  unsigned long long n_analyses = 0;
  DevBuf<double> theta, base_g, X, A, mu, K, nu, S, P, eps, xi, yobs;
  DevBuf<int> bad;
  std::vector<std::unique_ptr<dbnet>> views;
};

namespace {

template <class F>
int ens_guard(dbens* h, F&& f) {
  try {
    f();
    return DBNET_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    if (h && h->eng && e.code == DBNET_ECUDA) {
      h->eng->poisoned = true;
      h->eng->poison_msg = e.msg;
    }
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return DBNET_ENOMEM;
  } catch (...) {
    g_last_error = "unexpected failure";
    return DBNET_ECUDA;
  }
}

int resolve_target(const dbens_enkf_t& k, int slot) {
  if (k.target[slot] != DBENS_T_DEFAULT) return k.target[slot];
  return slot == 0 ? DBENS_T_AMPA : DBENS_T_GABA_A;
}

double target_value(const dbnet_region_params_t& p, int target) {
  if (target == DBENS_T_IEXT) return p.I_ext;
  if (target >= DBENS_T_AMPA && target <= DBENS_T_GABA_B) return p.g_u[target - DBENS_T_AMPA];
  return 0.0;
}

void scale_target(dbnet_region_params_t& p, int target, double v) {
  if (target == DBENS_T_IEXT) p.I_ext = v;
  else if (target >= DBENS_T_AMPA && target <= DBENS_T_GABA_B) p.g_u[target - DBENS_T_AMPA] = v;
}

void check_enkf(const dbens_enkf_t& k) {
  if (!(k.obs_var > 0) || !std::isfinite(k.obs_var)) raise(DBNET_EINVAL, "obs_var must be > 0");
  if (!(k.gamma >= 0 && k.gamma <= 1)) raise(DBNET_EINVAL, "gamma must be in [0, 1]");
  if (!(k.rw_sigma >= 0) || !std::isfinite(k.rw_sigma)) raise(DBNET_EINVAL, "rw_sigma must be >= 0");
  if (!(k.theta_lo <= k.theta_hi) || !std::isfinite(k.theta_lo) || !std::isfinite(k.theta_hi))
    raise(DBNET_EINVAL, "theta bounds must be finite with lo <= hi");
  for (int sl = 0; sl < 2; ++sl)
    if (k.target[sl] < DBENS_T_NONE || k.target[sl] > DBENS_T_IEXT)
      raise(DBNET_EINVAL, "target must be one of DBENS_T_*");
  const int a = resolve_target(k, 0), b = resolve_target(k, 1);
  if (a == b && a != DBENS_T_NONE) raise(DBNET_EINVAL, "the two log scales need distinct targets");
  if (!(k.floor > 0)) raise(DBNET_EINVAL, "floor must be > 0");
  if (k.mode != DBENS_DIFFUSION && k.mode != DBENS_GLOBAL) raise(DBNET_EINVAL, "unknown EnKF mode");
}

}  // namespace

extern "C" {

int ens_create(const dbnet_graph_t* graph, const dbnet_region_params_t* base, int32_t n_members,
               const double* log_scale_init, const dbnet_options_t* options,
               const dbens_enkf_t* enkf, void* cuda_stream, dbens_t** out) {
  if (out) *out = nullptr;
  std::unique_ptr<dbens> h(new (std::nothrow) dbens());
  if (!h) return DBNET_ENOMEM;
  int rc = ens_guard(nullptr, [&] {
    AllocStreamScope alloc_stream(cuda_stream);
    if (!out || !graph || !base || !log_scale_init || !options || !enkf)
      raise(DBNET_EINVAL, "NULL argument");
    if (n_members < 2) raise(DBNET_EINVAL, "an ensemble needs at least 2 members");
    check_options(*options);
    check_enkf(*enkf);
    const int R = graph->n_regions;
    if (R < 1) raise(DBNET_EINVAL, "n_regions must be >= 1");
    for (int r = 0; r < R; ++r) check_params(base[r], options->dt_ms, bin_lead(*options));
    const int M = n_members;
    for (int64_t i = 0; i < (int64_t)M * R * 2; ++i)
      if (!std::isfinite(log_scale_init[i])) raise(DBNET_EINVAL, "non-finite initial log scale");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    auto g = upload_graph(graph, s);
    std::vector<InstSpec> specs((size_t)M);
    for (int m = 0; m < M; ++m) {
      InstSpec& sp = specs[(size_t)m];
      sp.graph = g;
      sp.params.assign(base, base + R);
      for (int r = 0; r < R; ++r) {
        const double* t = log_scale_init + ((size_t)m * R + r) * 2;
        const double ta = std::min(std::max(t[0], enkf->theta_lo), enkf->theta_hi);
        const double tg = std::min(std::max(t[1], enkf->theta_lo), enkf->theta_hi);
        scale_target(sp.params[(size_t)r], resolve_target(*enkf, 0),
                     target_value(base[r], resolve_target(*enkf, 0)) * std::exp(ta));
        scale_target(sp.params[(size_t)r], resolve_target(*enkf, 1),
                     target_value(base[r], resolve_target(*enkf, 1)) * std::exp(tg));
      }
      sp.opt = *options;
      sp.net_id = options->net_id + (uint64_t)m;
    }
    h->eng.reset(new Engine());
    h->eng->init(specs, cuda_stream);
    h->M = M;
    h->R = R;
    h->enkf = *enkf;
    h->seed = options->seed;
    h->net_id0 = options->net_id;
    const int n = kB * R;
    h->theta.alloc((int64_t)M * R * 2);
    h->base_g.alloc((int64_t)R * 2);
    h->X.alloc((int64_t)M * n);
    h->A.alloc((int64_t)M * n);
    h->mu.alloc(n);
    h->K.alloc((int64_t)R * n);
    h->nu.alloc((int64_t)M * R);
    h->S.alloc((int64_t)R * R);
    h->P.alloc((int64_t)R * n);
    h->eps.alloc((int64_t)M * R);
    h->xi.alloc((int64_t)M * R * 2);
    h->yobs.alloc(R);
    h->bad.alloc(1);
    std::vector<double> th((size_t)M * R * 2), bg((size_t)R * 2);
    for (size_t i = 0; i < th.size(); ++i)
      th[i] = std::min(std::max(log_scale_init[i], enkf->theta_lo), enkf->theta_hi);
    h->target[0] = resolve_target(*enkf, 0);
    h->target[1] = resolve_target(*enkf, 1);
    for (int r = 0; r < R; ++r) {
      bg[2 * r] = target_value(base[r], h->target[0]);
      bg[2 * r + 1] = target_value(base[r], h->target[1]);
    }
    Engine& e = *h->eng;
    CK(cudaMemcpyAsync(h->theta.p, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, e.stream));
    CK(cudaMemcpyAsync(h->base_g.p, bg.data(), sizeof(double) * bg.size(), cudaMemcpyHostToDevice, e.stream));
    CK(cudaStreamSynchronize(e.stream));
  });
  if (rc == DBNET_OK) *out = h.release();
  return rc;
}

int ens_step(dbens_t* h, int64_t n_steps) {
  if (!h || !h->eng) return DBNET_EINVAL;
  return ens_guard(h, [&] { h->eng->step(n_steps); });
}

int ens_assimilate(dbens_t* h, const double* y_obs, const double* eps_obs, const double* xi_rw,
                   double* y_pred_mean) {
  if (!h || !h->eng || !y_obs) return DBNET_EINVAL;
  return ens_guard(h, [&] {
    Engine& e = *h->eng;
    e.sync();
    const int M = h->M, R = h->R, n = kB * R;
    for (int r = 0; r < R; ++r)
      if (!std::isfinite(y_obs[r])) raise(DBNET_EINVAL, "non-finite observation");
    for (int64_t i = 0; eps_obs && i < (int64_t)M * R; ++i)
      if (!std::isfinite(eps_obs[i])) raise(DBNET_EINVAL, "non-finite observation perturbation");
    for (int64_t i = 0; xi_rw && i < (int64_t)M * R * 2; ++i)
      if (!std::isfinite(xi_rw[i])) raise(DBNET_EINVAL, "non-finite random-walk draw");
    cudaStream_t s = e.stream;
    CK(cudaMemcpyAsync(h->yobs.p, y_obs, sizeof(double) * R, cudaMemcpyHostToDevice, s));
    if (eps_obs)
      CK(cudaMemcpyAsync(h->eps.p, eps_obs, sizeof(double) * M * R, cudaMemcpyHostToDevice, s));
    else
      k_normals<<<blocks(M * R), 128, 0, s>>>(h->eps.p, M * R, h->seed, h->net_id0, h->n_analyses, 2);
    if (xi_rw)
      CK(cudaMemcpyAsync(h->xi.p, xi_rw, sizeof(double) * M * R * 2, cudaMemcpyHostToDevice, s));
    else
      k_normals<<<blocks(M * R * 2), 128, 0, s>>>(h->xi.p, M * R * 2, h->seed, h->net_id0, h->n_analyses, 3);
    CK(cudaMemsetAsync(h->bad.p, 0, sizeof(int), s));
    k_gather<<<blocks(M * R), 128, 0, s>>>(h->X.p, h->theta.p, e.bw.p, e.ylast.p, M, R);
    k_mean_dev<<<blocks(n), 128, 0, s>>>(h->X.p, h->mu.p, h->A.p, M, n);
    const double G = h->enkf.obs_var, sd = std::sqrt(h->enkf.obs_var);
    k_innovation<<<blocks(M * R), 128, 0, s>>>(h->nu.p, h->X.p, h->yobs.p, h->eps.p, M, R, sd);
    if (h->enkf.mode == DBENS_DIFFUSION) {
      k_gain_diffusion<<<blocks(R * n), 128, 0, s>>>(h->A.p, h->K.p, M, n, R, G);
      k_fuse<<<blocks(M * n), 128, 0, s>>>(h->X.p, h->K.p, h->nu.p, M, R, h->enkf.gamma);
    } else {
      k_cov_obs<<<blocks(std::max(R * R, R * n)), 128, 0, s>>>(h->A.p, h->S.p, h->P.p, M, R, G);
      k_cholesky<<<1, 256, 0, s>>>(h->S.p, R, h->bad.p);
      k_chol_solve<<<blocks(n), 128, 0, s>>>(h->S.p, h->P.p, R, n);
      k_apply_global<<<blocks(M * n), 128, 0, s>>>(h->X.p, h->P.p, h->nu.p, M, R);
    }
    k_check_finite<<<blocks((int64_t)M * n), 128, 0, s>>>(h->X.p, (int64_t)M * n, h->bad.p);
    k_constrain_writeback<<<blocks(M * R), 128, 0, s>>>(h->X.p, h->theta.p, e.bw.p, M, R,
                                                         h->enkf.theta_lo, h->enkf.theta_hi,
                                                         h->enkf.floor, h->bad.p);
    k_walk_rescale<<<blocks(M * R), 128, 0, s>>>(h->theta.p, h->xi.p, h->base_g.p, e.desc.p, M, R,
                                                  h->enkf.rw_sigma, h->enkf.theta_lo, h->enkf.theta_hi,
                                                  h->target[0], h->target[1], h->bad.p);
    CK(cudaGetLastError());
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, h->bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    std::vector<double> mu;
    if (y_pred_mean) {
      mu.resize((size_t)n);
      CK(cudaMemcpyAsync(mu.data(), h->mu.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    h->n_analyses += 1;
    if (bad & 1) raise(DBNET_EINVAL, "observation covariance is not positive definite; members unchanged");
    if (bad) raise(DBNET_EINVAL, "the analysis produced a non-finite state; members unchanged");
    if (y_pred_mean)
      for (int r = 0; r < R; ++r) y_pred_mean[r] = mu[(size_t)(kB * r + kY)];
  });
}

int ens_read(dbens_t* h, double* theta, double* bw, double* y) {
  if (!h || !h->eng) return DBNET_EINVAL;
  return ens_guard(h, [&] {
    Engine& e = *h->eng;
    e.sync();
    const int64_t MR = (int64_t)h->M * h->R;
    if (theta) CK(cudaMemcpy(theta, h->theta.p, sizeof(double) * MR * 2, cudaMemcpyDeviceToHost));
    if (bw) CK(cudaMemcpy(bw, e.bw.p, sizeof(double) * MR * 4, cudaMemcpyDeviceToHost));
    if (y) CK(cudaMemcpy(y, e.ylast.p, sizeof(double) * MR, cudaMemcpyDeviceToHost));
  });
}

int ens_member(dbens_t* h, int32_t member, dbnet_t** out) {
  if (!h || !h->eng || !out || member < 0 || member >= h->M) return DBNET_EINVAL;
  return ens_guard(h, [&] {
    if (h->views.empty()) h->views.resize((size_t)h->M);
    auto& v = h->views[(size_t)member];
    if (!v) {
      v.reset(new dbnet());
      v->eng = h->eng.get();
      v->inst = member;
    }
    *out = v.get();
  });
}

void ens_destroy(dbens_t* h) { delete h; }

}  // extern "C"

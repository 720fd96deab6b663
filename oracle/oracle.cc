// CPU oracle for the Digital Brain hot path.  TEST INFRASTRUCTURE ONLY: the
// tests, the smoke check and the benchmark's CPU-baseline leg may call it; the
// product (the CUDA library) never does, and the two share no code.
//
// It is a plain, slow restatement of the method, step by step, in the order
// the paper gives it (single-threaded; an optional timing variant, set by
// og_set_threads, runs the neuron loop over contiguous ranges on several
// threads and the delivery with atomic integer additions, with results
// identical to the single-threaded loop):
//   * conductance LIF neurons (Methods, "Simulating Digital Brain on GPUs",
//     the capacitance-voltage equation and Eq. 2; Supplementary Sec. 3,
//     "Numerical method", Eqs. 3 and 5 with the refractory reset);
//   * push-based spike delivery (Supplementary Algorithm 2) into a ring of
//     per-delay integer accumulators, indexed [slot][neuron][class] (or
//     [slot][neuron][channel] with two weights per edge);
//   * Poisson background input (Extended Data Table 2, "Input");
//   * per-region spike counts and the Balloon-Windkessel BOLD model
//     (Extended Data Table 4), integrated by forward Euler in FP64.
// The neuron arithmetic is a template over the state type: `double` is the
// FP64 oracle, `float` is the op-order-matched FP32 oracle whose every
// operation is written out below in the order the CUDA path must follow.
// Build with -ffp-contract=off so no multiply-add is fused.
//
// Readings of the paper where it is silent or garbled (each also listed in
// the design notes):
//   * Eq. 5 omits 1/C and the step on the background term: the whole bracket
//     is multiplied by dt/C, as the capacitance-voltage equation implies.
//   * Eq. 5 uses J(t) and V(t): V is advanced with the pre-update J, then J.
//   * A spike is registered when the advanced V reaches V_th (>=); V is then
//     set to V_reset and held there for round(T_ref/dt) further steps while J
//     keeps integrating.
//   * Delays: an edge with delay d >= 1 carries a spike emitted at step n into
//     the accumulator read at step n+d (d = 1 is Eq. 3's one-step latency).
//   * One weight per edge, shared by both channels of the source's class, so
//     the accumulator has two classes: E (AMPA, NMDA) and I (GABA_A, GABA_B).
//     Optionally a second weight per edge, as the connection table of
//     Supplementary Table 5 stores one weight per channel: the first feeds
//     AMPA (excitatory source) or GABA_A (inhibitory), the second NMDA or
//     GABA_B, and the accumulator has the four channels.  The background
//     drive then adds w_ext to both AMPA and NMDA, as it adds to E in the
//     one-weight form.
//   * Accumulators hold fixed point: q(w) = rint(w * 2^S).
//   * Optional spike binning (Supplementary Sec. 3, "Numerical method"): the
//     accumulated spike A_j(t) is non-zero only at bin edges t = k b_t, where
//     it marks a spike of j in (t - b_t, t].  A spike of any step of a bin is
//     handed on as if emitted in the bin's last step; a neuron that fires
//     twice in one bin is handed on once (A_j is 0 or 1).
//   * Weights are the BF16 values the device stores.  Optionally the first
//     weight is an unrounded FP64 value instead (still accumulated as
//     rint(w * 2^S), an absolute error of at most 2^-(S+1)), which states
//     what the BF16 rounding of the weights costs.
//   * Background: K_ext independent Poisson sources of rate nu per neuron,
//     each adding w_ext to the E class; the count per step is drawn by integer
//     inversion of one 32-bit Philox word against FP64 Poisson CDF thresholds.
//   * z (neural activity) = z_scale * spikes of the region in the last bin /
//     region size; BW constants are inputs.
//   * Optional background current I_bg (Eq. 1; Extended Data Table 2, "OU
//     current"): Eq. 4 prints the noise as sqrt(2 tau) sigma eps with no
//     step; the Euler-Maruyama form of Eq. 1 is used instead,
//     I_bg += (mu - I_bg) dt/tau + sigma sqrt(2 dt/tau) xi, whose stationary
//     standard deviation is sigma.  V is advanced with the old I_bg (added
//     after I_ext, inside the dt/C bracket), then I_bg.  I_bg starts at mu.
//     xi is a standard normal by the Box-Muller transform of the neuron's
//     Philox word of stream 4: u1 = (high 32 bits + 1) 2^-32, u2 = low 32
//     bits 2^-32, xi = sqrt(-2 ln u1) cos(2 pi u2), in FP64 (host and device
//     log/cos differ, so with sigma > 0 only the FP64 results are meant to
//     be compared, statistically).
//   * Heterogeneous injected current (Methods: the I_ext,i are Gamma
//     distributed with region hyperparameters): with a region shape k > 0,
//     neuron i receives I_ext * G_i / k, G_i ~ Gamma(k, 1) drawn once by the
//     Marsaglia-Tsang method (ACM TOMS 26(3), 2000) from its Philox words of
//     stream 5 (attempt a uses counter (0, i, 5, a): word 0 a Box-Muller
//     normal, word 1 the acceptance uniform, word 2 for k < 1 the uniform of
//     G(k) = G(k + 1) U^(1/k)), in FP64, rounded once to the state type.
#include <omp.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplications with the
// published multipliers, the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ull * x0;
    unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ull * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// The 64-bit word that neuron i draws at step n from stream `stream`:
// counter (n, floor(i/4), stream, 0), key (seed, net_id), word i mod 4.
uint64_t neuron_word(uint64_t seed, uint64_t net_id, uint64_t n, int64_t i, uint64_t stream) {
  uint64_t ctr[4] = {n, (uint64_t)(i >> 2), stream, 0};
  uint64_t key[2] = {seed, net_id};
  uint64_t out[4];
  philox4x64_10(ctr, key, out);
  return out[i & 3];
}

double bf16_value(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

}  // namespace

extern "C" {

struct OgGraph {
  int32_t n_neurons, n_regions;
  const int32_t* region_offsets;  // [R+1]
  const int32_t* n_exc;           // [R]
  const int64_t* row_ptr;         // [N+1], CSR by source
  const int32_t* col;             // [E] target
  const uint16_t* w_bf16;         // [E]
  const uint8_t* delay;           // [E] steps >= 1
  const uint16_t* w2_bf16;        // [E] second channel's weight, or NULL (one weight)
  const double* w_f64;            // [E] unrounded first weight, or NULL (w_bf16 is used)
};

struct OgRegion {  // units: mV, ms, nF, uS, nA
  double C, gL, VL, Vth, Vreset, Tref;
  double Vu[4], tau_u[4], g_u[4];
  double I_ext, drive_rate_hz, drive_K, w_ext;
  double ou_mu, ou_sigma, ou_tau;  // background OU current; off when mu = sigma = 0
  double iext_shape;               // > 0: per-neuron I_ext factor G/k, G ~ Gamma(k, 1)
};

struct OgOptions {
  double dt_ms, bin_ms, tr_ms, z_scale;
  double bw_kappa, bw_gamma, bw_tau, bw_alpha, bw_rho, bw_V0;
  uint64_t seed, net_id;
  int32_t fixed_shift;  // 0 = automatic
  int32_t precision;    // 32 = matched FP32, 64 = FP64
  int32_t bin_spikes;   // 1: spikes are handed on at the end of their bin
  int32_t pad;
};

void og_philox4x64_10(const uint64_t* ctr, const uint64_t* key, uint64_t* out) {
  philox4x64_10(ctr, key, out);
}

// Poisson CDF thresholds for the integer-inversion drive: thr[k] =
// floor(P(X <= k) * 2^32) for the leading k whose value stays below 2^32
// (at most 16).  A draw u (32 bits) gives the count #{k : u >= thr[k]}.
int32_t og_poisson_thresholds(double lam, uint32_t* thr) {
  if (!(lam >= 0.0)) return -1;
  double p = std::exp(-lam);
  double cdf = p;
  int32_t n = 0;
  for (int32_t k = 0; k < 16; ++k) {
    double t = std::floor(std::ldexp(cdf, 32));
    if (t >= 4294967296.0) break;
    thr[k] = (uint32_t)t;
    n = k + 1;
    p = p * lam;
    p = p / (double)(k + 1);
    cdf = cdf + p;
  }
  return n;
}

// Forward-Euler step of the Balloon-Windkessel model (Extended Data Table 4)
// for one region: state x = (s, f, v, q), neural activity z, step h seconds.
// Returns the BOLD signal of the advanced state.
double og_bw_step(double* x, double z, double h, double kappa, double gamma, double tau,
                  double alpha, double rho, double V0) {
  double s = x[0], f = x[1], v = x[2], q = x[3];
  double fout = std::pow(v, 1.0 / alpha);
  double E = 1.0 - std::pow(1.0 - rho, 1.0 / f);
  double ds = z - kappa * s - gamma * (f - 1.0);
  double df = s;
  double dv = (f - fout) / tau;
  double dq = (f * E / rho - fout * q / v) / tau;
  x[0] = s + h * ds;
  x[1] = f + h * df;
  x[2] = v + h * dv;
  x[3] = q + h * dq;
  double k1 = 7.0 * rho, k2 = 2.0, k3 = 2.0 * rho - 0.2;
  return V0 * (k1 * (1.0 - x[3]) + k2 * (1.0 - x[3] / x[2]) + k3 * (1.0 - x[2]));
}

}  // extern "C"

namespace {

template <class Real>
struct RegionConst {
  Real dtC, gL, VL, Vth, Vreset, Iext;
  Real g[4], Vu[4], dec[4];
  int32_t n_ref, q_ext, n_thr;
  uint32_t thr[16];
  int32_t ou_on;
  Real ou_mu, ou_k, ou_s;  // mu, dt/tau, sigma sqrt(2 dt/tau)
  int32_t het;             // per-neuron I_ext factors
};

// A uniform in (0, 1] from the high half of a Philox word.
double unit_open(uint64_t w) { return ((double)(w >> 32) + 1.0) * std::ldexp(1.0, -32); }

// Standard normal from one 64-bit Philox word (Box-Muller, FP64).
double box_muller(uint64_t w) {
  const double u1 = ((double)(w >> 32) + 1.0) * std::ldexp(1.0, -32);  // (0, 1]
  const double u2 = (double)(w & 0xFFFFFFFFull) * std::ldexp(1.0, -32);  // [0, 1)
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.14159265358979323846 * u2);
}

// Gamma(k, 1) for neuron i from its stream-5 Philox words (Marsaglia-Tsang).
double gamma_draw(double k, uint64_t seed, uint64_t net_id, int64_t i) {
  const uint64_t key[2] = {seed, net_id};
  const double kk = k < 1.0 ? k + 1.0 : k;
  const double d = kk - 1.0 / 3.0;
  const double c = 1.0 / std::sqrt(9.0 * d);
  for (uint64_t a = 0;; ++a) {
    const uint64_t ctr[4] = {0, (uint64_t)i, 5, a};
    uint64_t w[4];
    philox4x64_10(ctr, key, w);
    const double x = box_muller(w[0]);
    const double t = 1.0 + c * x;
    if (t <= 0.0) continue;
    const double v = t * t * t;
    const double u = unit_open(w[1]);
    if (std::log(u) < 0.5 * x * x + d - d * v + d * std::log(v)) {
      double g = d * v;
      if (k < 1.0) g = g * std::pow(unit_open(w[2]), 1.0 / k);
      return g;
    }
  }
}

struct SimBase {
  virtual ~SimBase() {}
  virtual void step(int64_t n_steps) = 0;
  virtual void deliver_only(const int32_t* ids, int64_t count, int64_t n) = 0;
  virtual void read_state(double* V, double* J, int32_t* ref) const = 0;
  virtual void set_state(const double* V, const double* J, const int32_t* ref) = 0;
  virtual void read_ibg(double* I) const = 0;
  virtual void set_ibg(const double* I) = 0;
  // shared bookkeeping
  int32_t N = 0, R = 0, D = 0, S = 0, spb = 0, bins_per_tr = 0;
  int32_t nch = 2;  // accumulator channels: 2 classes, or 4 with two weights per edge
  int32_t threads = 1;  // > 1: the timing variant (OpenMP), same results
  int32_t bin_spikes = 0;
  int64_t n = 0, events = 0, spikes = 0, bins_done = 0;
  std::vector<int64_t> last_release;  // with bin_spikes: release step of each neuron's last spike
  std::vector<int64_t> ring;  // [D][N][nch]
  std::vector<int32_t> raster_step, raster_id;
  std::vector<int32_t> region_of, cnt;
  std::vector<double> bw;    // [R][4]
  std::vector<double> bold;  // [samples][R]
};

template <class Real>
struct Sim : SimBase {
  OgGraph g;
  OgOptions o;
  std::vector<RegionConst<Real>> rc;
  std::vector<int32_t> n_exc_end;  // absolute index where the inhibitory block starts
  std::vector<Real> V, J;  // J as [4][N]
  std::vector<int32_t> ref;
  std::vector<Real> Ibg;   // background OU current
  std::vector<Real> fext;  // per-neuron I_ext factor (1 where homogeneous)

  int32_t class_of(int32_t i) const {
    int32_t r = region_of[(size_t)i];
    return i < n_exc_end[(size_t)r] ? 0 : 1;
  }

  // Supplementary Algorithm 2, the push of a spike's synaptic input: every
  // out-edge of spiker j adds q(w) to the accumulator slot its delay selects
  // (with two weights: q(w) to channel 2c and q(w2) to channel 2c + 1).
  // (The threaded timing variant adds with atomic integer additions: the sums
  // are exact, so their order does not matter.)
  static void add(int64_t& a, int64_t q, bool atomic) {
    if (atomic) __atomic_fetch_add(&a, q, __ATOMIC_RELAXED);
    else a += q;
  }
  int64_t scatter(int32_t j, int64_t step_n, bool atomic = false) {
    int32_t c = class_of(j);
    int64_t ev = 0;
    for (int64_t e = g.row_ptr[j]; e < g.row_ptr[j + 1]; ++e) {
      int64_t slot = (step_n + g.delay[e]) % D;
      double w = g.w_f64 ? g.w_f64[e] : bf16_value(g.w_bf16[e]);
      int64_t q = (int64_t)std::lrint(std::ldexp(w, S));
      if (nch == 2) {
        add(ring[(size_t)((slot * N + g.col[e]) * 2 + c)], q, atomic);
      } else {
        int64_t q2 = (int64_t)std::lrint(std::ldexp(bf16_value(g.w2_bf16[e]), S));
        add(ring[(size_t)((slot * N + g.col[e]) * 4 + 2 * c)], q, atomic);
        add(ring[(size_t)((slot * N + g.col[e]) * 4 + 2 * c + 1)], q2, atomic);
      }
      ++ev;
    }
    return ev;
  }

  // The step at which a spike of step m is handed on.  Without binning it
  // is m itself.  With binning (Supplementary Sec. 3, "Numerical method": the
  // accumulated spike A_j(t) is non-zero only at bin edges t = k b_t and
  // then counts the spikes of (t - b_t, t]) a spike emitted in a step of the
  // bin [k spb, (k + 1) spb) takes effect as if emitted in the bin's last
  // step, so that an edge of delay d reaches the accumulator consumed at
  // step (k + 1) spb - 1 + d: with d = 1, the first step of the next bin.
  int64_t release_step(int64_t m) const {
    return bin_spikes ? (m / spb + 1) * spb - 1 : m;
  }

  // The spikes of one step, in neuron order: each is handed on to its
  // targets (once per bin with binning: A_j is an indicator).
  void deliver_fired(const std::vector<int32_t>& fired, int64_t step_n) {
    const int64_t rel = release_step(step_n);
    std::vector<int32_t> go;
    go.reserve(fired.size());
    for (int32_t j : fired) {
      if (bin_spikes) {
        if (last_release[(size_t)j] == rel) continue;
        last_release[(size_t)j] = rel;
      }
      go.push_back(j);
    }
    if (threads <= 1) {
      for (int32_t j : go) events += scatter(j, rel);
      return;
    }
    int64_t ev = 0;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 16) reduction(+ : ev)
    for (int64_t k = 0; k < (int64_t)go.size(); ++k) ev += scatter(go[(size_t)k], rel, true);
    events += ev;
  }

  void deliver_only(const int32_t* ids, int64_t count, int64_t step_n) override {
    for (int64_t k = 0; k < count; ++k) events += scatter(ids[k], step_n);
  }

  // One neuron's step (the order of operations the matched-FP32 oracle fixes).
  void update_neuron(int32_t i, int64_t slot, Real inv2S, std::vector<int32_t>& fired) {
    const RegionConst<Real>& p = rc[(size_t)region_of[(size_t)i]];
    // this step's arrivals per channel (AMPA, NMDA, GABA_A, GABA_B): in
    // the one-weight form both channels of a class read its class sum
    int64_t* a = &ring[(size_t)((slot * N + i) * nch)];
    int64_t ach[4];
    for (int u4 = 0; u4 < 4; ++u4) ach[u4] = nch == 2 ? a[u4 / 2] : a[u4];
    for (int k = 0; k < nch; ++k) a[k] = 0;
    // background Poisson count by integer inversion
    uint32_t u = (uint32_t)(neuron_word(o.seed, o.net_id, (uint64_t)n, i, 0) >> 32);
    int64_t c = 0;
    for (int32_t k = 0; k < p.n_thr; ++k) c += (u >= p.thr[k]) ? 1 : 0;
    ach[0] += c * (int64_t)p.q_ext;
    ach[1] += c * (int64_t)p.q_ext;
    // membrane (Eq. 5, bracket times dt/C) with the old V and J
    Real v = V[(size_t)i];
    Real Isyn = (Real)0;
    for (int u4 = 0; u4 < 4; ++u4) {
      Real gj = p.g[u4] * J[(size_t)u4 * N + i];
      Real dv = p.Vu[u4] - v;
      Real t = gj * dv;
      Isyn = Isyn + t;
    }
    Real leak = p.gL * (v - p.VL);
    Real I = Isyn - leak;
    if (p.het) {
      Real ie = p.Iext * fext[(size_t)i];
      I = I + ie;
    } else {
      I = I + p.Iext;
    }
    if (p.ou_on) I = I + Ibg[(size_t)i];
    Real dV = I * p.dtC;
    Real vn = v + dV;
    // background current (Eq. 1, Euler-Maruyama) after its use above
    if (p.ou_on) {
      Real& ib = Ibg[(size_t)i];
      const Real xi = (Real)box_muller(neuron_word(o.seed, o.net_id, (uint64_t)n, i, 4));
      Real dI = p.ou_mu - ib;
      Real t1 = dI * p.ou_k;
      ib = ib + t1;
      Real t2 = p.ou_s * xi;
      ib = ib + t2;
    }
    // synaptic traces (Eq. 3): decay, then this step's arrivals
    for (int u4 = 0; u4 < 4; ++u4) {
      Real x = (Real)ach[u4] * inv2S;
      Real& j = J[(size_t)u4 * N + i];
      Real d = p.dec[u4] * j;
      j = d + x;
    }
    // refractory clamp, threshold and reset
    if (ref[(size_t)i] > 0) {
      V[(size_t)i] = p.Vreset;
      ref[(size_t)i] -= 1;
    } else if (vn >= p.Vth) {
      V[(size_t)i] = p.Vreset;
      ref[(size_t)i] = p.n_ref;
      fired.push_back(i);
    } else {
      V[(size_t)i] = vn;
    }
  }

  void step(int64_t n_steps) override {
    const Real inv2S = (Real)std::ldexp(1.0, -S);
    for (int64_t it = 0; it < n_steps; ++it, ++n) {
      const int64_t slot = n % D;
      std::vector<int32_t> fired;
      if (threads <= 1) {
        for (int32_t i = 0; i < N; ++i) update_neuron(i, slot, inv2S, fired);
      } else {
        // timing variant: contiguous neuron ranges per thread, their spike
        // lists joined in neuron order (the same list as the loop above)
        std::vector<std::vector<int32_t>> part((size_t)threads);
#pragma omp parallel num_threads(threads)
        {
          const int t = omp_get_thread_num();
          const int32_t lo = (int32_t)((int64_t)N * t / threads);
          const int32_t hi = (int32_t)((int64_t)N * (t + 1) / threads);
          for (int32_t i = lo; i < hi; ++i) update_neuron(i, slot, inv2S, part[(size_t)t]);
        }
        for (auto& v : part) fired.insert(fired.end(), v.begin(), v.end());
      }
      deliver_fired(fired, n);
      for (int32_t j : fired) {
        raster_step.push_back((int32_t)n);
        raster_id.push_back(j);
        cnt[(size_t)region_of[(size_t)j]] += 1;
        ++spikes;
      }
      // bin end: neural activity into the hemodynamic model
      if ((n + 1) % spb == 0) {
        const double h = o.bin_ms * 1e-3;
        std::vector<double> y((size_t)R);
        for (int32_t r = 0; r < R; ++r) {
          double nr = (double)(g.region_offsets[r + 1] - g.region_offsets[r]);
          double z = o.z_scale * (double)cnt[(size_t)r] / nr;
          cnt[(size_t)r] = 0;
          y[(size_t)r] = og_bw_step(&bw[(size_t)r * 4], z, h, o.bw_kappa, o.bw_gamma, o.bw_tau,
                                    o.bw_alpha, o.bw_rho, o.bw_V0);
        }
        ++bins_done;
        if (bins_done % bins_per_tr == 0) bold.insert(bold.end(), y.begin(), y.end());
      }
    }
  }

  void read_state(double* Vo, double* Jo, int32_t* refo) const override {
    for (int32_t i = 0; i < N; ++i) {
      if (Vo) Vo[i] = (double)V[(size_t)i];
      if (refo) refo[i] = ref[(size_t)i];
      for (int u = 0; u < 4 && Jo; ++u) Jo[(size_t)u * N + i] = (double)J[(size_t)u * N + i];
    }
  }

  void read_ibg(double* I) const override {
    for (int32_t i = 0; i < N; ++i) I[i] = (double)Ibg[(size_t)i];
  }
  void set_ibg(const double* I) override {
    for (int32_t i = 0; i < N; ++i) Ibg[(size_t)i] = (Real)I[i];
  }

  void set_state(const double* Vi, const double* Ji, const int32_t* refi) override {
    for (int32_t i = 0; i < N; ++i) {
      if (Vi) V[(size_t)i] = (Real)Vi[i];
      if (refi) ref[(size_t)i] = refi[i];
      for (int u = 0; u < 4 && Ji; ++u) J[(size_t)u * N + i] = (Real)Ji[(size_t)u * N + i];
    }
  }
};

template <class Real>
SimBase* make_sim(const OgGraph* g, const OgRegion* regs, const OgOptions* o, int* err) {
  auto* s = new Sim<Real>();
  s->g = *g;
  s->o = *o;
  const int32_t N = g->n_neurons, R = g->n_regions;
  s->N = N;
  s->R = R;
  // ring depth: longest delay + 1
  int32_t dmax = 1, kin_max = 0;
  double wmax = 0.0;
  std::vector<int32_t> indeg((size_t)N, 0);
  for (int64_t e = 0; e < g->row_ptr[N]; ++e) {
    dmax = g->delay[e] > dmax ? g->delay[e] : dmax;
    double w = g->w_f64 ? g->w_f64[e] : bf16_value(g->w_bf16[e]);
    wmax = w > wmax ? w : wmax;
    if (g->w2_bf16) {
      double w2 = bf16_value(g->w2_bf16[e]);
      wmax = w2 > wmax ? w2 : wmax;
    }
    indeg[(size_t)g->col[e]] += 1;
  }
  for (int32_t i = 0; i < N; ++i) kin_max = indeg[(size_t)i] > kin_max ? indeg[(size_t)i] : kin_max;
  // with binning a spike waits up to spb - 1 steps for its bin to end
  const int32_t spb = (int32_t)std::lrint(o->bin_ms / o->dt_ms);
  s->bin_spikes = o->bin_spikes ? 1 : 0;
  s->D = dmax + 1 + (s->bin_spikes && spb > 1 ? spb - 1 : 0);
  double wext_max = 0.0;
  for (int32_t r = 0; r < R; ++r) wext_max = regs[r].w_ext > wext_max ? regs[r].w_ext : wext_max;
  // fixed-point scale: 2^S, S = 16 unless the worst-case sum of one step's
  // arrivals (every in-edge at the largest weight plus 16 background events)
  // would not fit in int32
  auto bound = [&](int32_t S) {
    return (double)kin_max * std::rint(std::ldexp(wmax, S)) + 16.0 * std::rint(std::ldexp(wext_max, S));
  };
  int32_t S = o->fixed_shift > 0 ? o->fixed_shift : 16;
  if (o->fixed_shift <= 0)
    while (S > 0 && bound(S) > 2147483647.0) --S;
  if (bound(S) > 2147483647.0) { *err = -5; delete s; return nullptr; }
  s->S = S;
  s->spb = (int32_t)std::lrint(o->bin_ms / o->dt_ms);
  s->bins_per_tr = (int32_t)std::lrint(o->tr_ms / o->bin_ms);
  if (s->spb < 1 || s->bins_per_tr < 1) { *err = -1; delete s; return nullptr; }
  s->region_of.resize((size_t)N);
  s->n_exc_end.resize((size_t)R);
  for (int32_t r = 0; r < R; ++r) {
    for (int32_t i = g->region_offsets[r]; i < g->region_offsets[r + 1]; ++i) s->region_of[(size_t)i] = r;
    s->n_exc_end[(size_t)r] = g->region_offsets[r] + g->n_exc[r];
  }
  s->rc.resize((size_t)R);
  for (int32_t r = 0; r < R; ++r) {
    const OgRegion& p = regs[r];
    RegionConst<Real>& c = s->rc[(size_t)r];
    c.dtC = (Real)(o->dt_ms / p.C);
    c.gL = (Real)p.gL;
    c.VL = (Real)p.VL;
    c.Vth = (Real)p.Vth;
    c.Vreset = (Real)p.Vreset;
    c.Iext = (Real)p.I_ext;
    for (int u = 0; u < 4; ++u) {
      c.g[u] = (Real)p.g_u[u];
      c.Vu[u] = (Real)p.Vu[u];
      c.dec[u] = (Real)std::exp(-o->dt_ms / p.tau_u[u]);
    }
    c.n_ref = (int32_t)std::lrint(p.Tref / o->dt_ms);
    c.q_ext = (int32_t)std::lrint(std::ldexp(p.w_ext, S));
    double lam = p.drive_K * p.drive_rate_hz * o->dt_ms * 1e-3;
    c.n_thr = og_poisson_thresholds(lam, c.thr);
    if (c.n_thr < 0) { *err = -1; delete s; return nullptr; }
    c.ou_on = (p.ou_mu != 0.0 || p.ou_sigma != 0.0) ? 1 : 0;
    if (c.ou_on && !(p.ou_tau > 0.0)) { *err = -1; delete s; return nullptr; }
    c.ou_mu = (Real)p.ou_mu;
    c.ou_k = c.ou_on ? (Real)(o->dt_ms / p.ou_tau) : (Real)0;
    c.ou_s = c.ou_on ? (Real)(p.ou_sigma * std::sqrt(2.0 * o->dt_ms / p.ou_tau)) : (Real)0;
    if (!(p.iext_shape >= 0.0)) { *err = -1; delete s; return nullptr; }
    c.het = p.iext_shape > 0.0 ? 1 : 0;
  }
  s->V.resize((size_t)N);
  s->J.assign((size_t)4 * N, (Real)0);
  s->ref.assign((size_t)N, 0);
  s->Ibg.resize((size_t)N);
  for (int32_t i = 0; i < N; ++i) s->Ibg[(size_t)i] = s->rc[(size_t)s->region_of[(size_t)i]].ou_mu;
  s->fext.assign((size_t)N, (Real)1);
  for (int32_t i = 0; i < N; ++i) {
    const double k = regs[s->region_of[(size_t)i]].iext_shape;
    if (k > 0.0) s->fext[(size_t)i] = (Real)(gamma_draw(k, o->seed, o->net_id, i) / k);
  }
  // initial V uniform in [V_reset, V_th) from the neuron's own Philox word
  for (int32_t i = 0; i < N; ++i) {
    const RegionConst<Real>& p = s->rc[(size_t)s->region_of[(size_t)i]];
    uint64_t w = neuron_word(o->seed, o->net_id, 0, i, 1);
    Real u = (Real)(w >> 40) * (Real)std::ldexp(1.0, -24);
    Real span = p.Vth - p.Vreset;
    Real t = span * u;
    s->V[(size_t)i] = p.Vreset + t;
  }
  s->nch = g->w2_bf16 ? 4 : 2;
  s->ring.assign((size_t)s->D * N * s->nch, 0);
  if (s->bin_spikes) s->last_release.assign((size_t)N, -1);
  s->cnt.assign((size_t)R, 0);
  s->bw.resize((size_t)R * 4);
  for (int32_t r = 0; r < R; ++r) {
    s->bw[(size_t)r * 4 + 0] = 0.0;
    s->bw[(size_t)r * 4 + 1] = 1.0;
    s->bw[(size_t)r * 4 + 2] = 1.0;
    s->bw[(size_t)r * 4 + 3] = 1.0;
  }
  *err = 0;
  return s;
}

}  // namespace

extern "C" {

void* og_create(const OgGraph* g, const OgRegion* regs, const OgOptions* o, int* err) {
  *err = -1;
  if (!g || !regs || !o || g->n_neurons <= 0 || g->n_regions <= 0) return nullptr;
  if (!(o->dt_ms > 0.0) || !(o->bin_ms > 0.0) || !(o->tr_ms > 0.0)) return nullptr;
  for (int64_t e = 0; e < g->row_ptr[g->n_neurons]; ++e)
    if (g->delay[e] < 1 || g->col[e] < 0 || g->col[e] >= g->n_neurons) { *err = -2; return nullptr; }
  if (o->precision == 64) return make_sim<double>(g, regs, o, err);
  if (o->precision == 32) return make_sim<float>(g, regs, o, err);
  return nullptr;
}

void og_destroy(void* h) { delete (SimBase*)h; }
// Threads of the timing variant (1 = the plain loop; results are identical).
void og_set_threads(void* h, int32_t n) { ((SimBase*)h)->threads = n > 1 ? n : 1; }
void og_step(void* h, int64_t n) { ((SimBase*)h)->step(n); }
void og_deliver_only(void* h, const int32_t* ids, int64_t count, int64_t n) {
  ((SimBase*)h)->deliver_only(ids, count, n);
}
void og_read_state(void* h, double* V, double* J, int32_t* ref) { ((SimBase*)h)->read_state(V, J, ref); }
void og_set_state(void* h, const double* V, const double* J, const int32_t* ref) {
  ((SimBase*)h)->set_state(V, J, ref);
}
void og_read_ibg(void* h, double* I) { ((SimBase*)h)->read_ibg(I); }
void og_set_ibg(void* h, const double* I) { ((SimBase*)h)->set_ibg(I); }
// the Box-Muller normal the OU current draws from a Philox word
double og_box_muller(uint64_t w) { return box_muller(w); }
// Gamma(k, 1) as drawn for neuron i's injected-current factor
double og_gamma_draw(double k, uint64_t seed, uint64_t net_id, int64_t i) {
  return gamma_draw(k, seed, net_id, i);
}

// info: [N, R, D, S, step, events, spikes, raster_len, bold_samples, bins_done]
void og_info(void* h, int64_t* info) {
  SimBase* s = (SimBase*)h;
  info[0] = s->N; info[1] = s->R; info[2] = s->D; info[3] = s->S; info[4] = s->n;
  info[5] = s->events; info[6] = s->spikes; info[7] = (int64_t)s->raster_id.size();
  info[8] = (int64_t)(s->bold.size() / (size_t)s->R); info[9] = s->bins_done;
}

void og_read_raster(void* h, int32_t* step, int32_t* id) {
  SimBase* s = (SimBase*)h;
  std::memcpy(step, s->raster_step.data(), s->raster_step.size() * 4);
  std::memcpy(id, s->raster_id.data(), s->raster_id.size() * 4);
}

void og_read_bold(void* h, double* y) {
  SimBase* s = (SimBase*)h;
  std::memcpy(y, s->bold.data(), s->bold.size() * 8);
}

void og_read_bw(void* h, double* x) {
  SimBase* s = (SimBase*)h;
  std::memcpy(x, s->bw.data(), s->bw.size() * 8);
}

void og_read_ring(void* h, int64_t* out) {
  SimBase* s = (SimBase*)h;
  std::memcpy(out, s->ring.data(), s->ring.size() * 8);
}

void og_read_counts(void* h, int32_t* out) {
  SimBase* s = (SimBase*)h;
  std::memcpy(out, s->cnt.data(), s->cnt.size() * 4);
}

}  // extern "C"

// Seeded synthetic network generator: the input side shared by the CPU oracle
// and the CUDA path.  It holds none of the simulation arithmetic -- it only
// draws graphs shaped like the networks the paper simulates:
//   * populations with a 4:1 excitatory/inhibitory split (Extended Data Table 2),
//   * a fixed in-degree per neuron, sources drawn uniformly without replacement,
//     no autapses and no multapses (Extended Data Table 2, "Connectivity"),
//   * a within-region share of the in-degree and a cross-region share whose
//     source region follows a row-stochastic region matrix, cross-region
//     sources being excitatory (long-range projections; Supplementary Sec. 2),
//   * lognormal weights rounded to BF16 and integer delays in steps.
// The output is a CSR by source whose rows are sorted by (delay, target).
//
// Every draw comes from a counter-based stream keyed by (seed, target), so
// the graph does not depend on the number of threads.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

inline uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Rng {
  uint64_t s;
  Rng(uint64_t seed, uint64_t stream, uint64_t sub) {
    s = seed ^ 0x6A09E667F3BCC909ull;
    splitmix64(s);
    s ^= stream * 0xD1B54A32D192ED03ull;
    splitmix64(s);
    s ^= sub * 0x8CB92BA72F3D8DD7ull;
    splitmix64(s);
  }
  uint64_t next() { return splitmix64(s); }
  // uniform integer in [0, n) by the multiply-high reduction
  uint32_t below(uint32_t n) {
    return (uint32_t)(((unsigned __int128)next() * n) >> 64);
  }
  double unit() {  // (0, 1]
    return ((next() >> 11) + 1) * (1.0 / 9007199254740992.0);
  }
  double normal() {
    double u1 = unit(), u2 = unit();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

inline uint16_t f32_to_bf16_rne(float f) {
  uint32_t b;
  std::memcpy(&b, &f, 4);
  b += 0x7FFFu + ((b >> 16) & 1u);
  return (uint16_t)(b >> 16);
}

}  // namespace

extern "C" {

struct SynthSpec {
  int32_t n_neurons;
  int32_t n_regions;
  const int32_t* region_offsets;  // [R+1], neurons sorted by region
  const int32_t* n_exc;           // [R], excitatory neurons first in each region
  int32_t k_in;                   // fixed in-degree
  int32_t k_within;               // of which drawn inside the target's region
  int32_t cross_exc_only;         // cross-region sources excitatory only
  int32_t d_within_min, d_within_max;  // delay range (steps) inside a region
  int32_t d_cross_min, d_cross_max;    // delay range (steps) across regions
  double w_mu, w_sigma;                // lognormal weight parameters
  const double* region_prob;           // [R*R] row-stochastic, diag ignored; may be NULL
  uint64_t seed;
};

// Region-to-region matrix: each off-diagonal entry is present with
// probability `density`, with a lognormal(mu, sigma) strength; rows are
// normalised to sum to one.  A row with no entry gets one at random.
int synth_region_matrix(int32_t R, double density, double mu, double sigma,
                        uint64_t seed, double* out) {
  if (R <= 0 || !out) return -1;
  for (int32_t r = 0; r < R; ++r) {
    Rng g(seed, 0xA11CEull, (uint64_t)r);
    double sum = 0.0;
    for (int32_t c = 0; c < R; ++c) {
      double v = 0.0;
      double u = g.unit();
      double s = std::exp(mu + sigma * g.normal());
      if (c != r && u <= density) v = s;
      out[(int64_t)r * R + c] = v;
      sum += v;
    }
    if (sum == 0.0 && R > 1) {
      int32_t c = (int32_t)g.below((uint32_t)(R - 1));
      if (c >= r) ++c;
      out[(int64_t)r * R + c] = 1.0;
      sum = 1.0;
    }
    for (int32_t c = 0; c < R; ++c)
      if (sum > 0.0) out[(int64_t)r * R + c] /= sum;
  }
  return 0;
}

}  // extern "C"

namespace {

// Draw the in-edges of one target.  The caller provides scratch: a bitmap
// sized for the largest region and a small open-addressing set for the
// cross-region sources.
struct TargetSampler {
  const SynthSpec& sp;
  std::vector<uint64_t> bitmap;
  std::vector<int32_t> chosen;
  std::vector<int32_t> hset;
  std::vector<size_t> used;
  const std::vector<std::vector<double>>& cdf;  // per region, over other regions

  TargetSampler(const SynthSpec& s, const std::vector<std::vector<double>>& c)
      : sp(s), cdf(c) {
    int32_t maxr = 0;
    for (int32_t r = 0; r < s.n_regions; ++r)
      maxr = std::max(maxr, s.region_offsets[r + 1] - s.region_offsets[r]);
    bitmap.assign((size_t)maxr / 64 + 1, 0ull);
    int hs = 16;
    while (hs < 4 * (s.k_in - s.k_within + 1)) hs <<= 1;
    hset.assign((size_t)hs, -1);
  }

  template <class F>
  void run(int32_t tgt, int32_t r, F&& emit) {
    Rng g(sp.seed, 0x7A6E7ull, (uint64_t)tgt);
    const int32_t r0 = sp.region_offsets[r], nr = sp.region_offsets[r + 1] - r0;
    const int32_t self = tgt - r0;
    const int32_t kw = sp.n_regions == 1 ? sp.k_in : sp.k_within;
    const int32_t kc = sp.k_in - kw;
    // Floyd's sampling of kw distinct values from the nr-1 non-self neurons
    chosen.clear();
    const int32_t m = nr - 1;
    for (int32_t j = m - kw; j < m; ++j) {
      int32_t t = (int32_t)g.below((uint32_t)j + 1);
      int32_t pick = (bitmap[t >> 6] >> (t & 63)) & 1ull ? j : t;
      bitmap[pick >> 6] |= 1ull << (pick & 63);
      chosen.push_back(pick);
    }
    for (int32_t c : chosen) {
      bitmap[c >> 6] &= ~(1ull << (c & 63));
      emit(r0 + (c < self ? c : c + 1), tgt, true);
    }
    if (kc <= 0) return;
    const size_t hmask = hset.size() - 1;
    used.clear();
    for (int32_t k = 0; k < kc; ++k) {
      int32_t src;
      for (;;) {
        double u = g.unit();
        const std::vector<double>& row = cdf[(size_t)r];
        int32_t rr = (int32_t)(std::lower_bound(row.begin(), row.end(), u) - row.begin());
        if (rr >= sp.n_regions) rr = sp.n_regions - 1;
        if (rr == r) continue;
        int32_t a = sp.region_offsets[rr];
        int32_t pool = sp.cross_exc_only ? sp.n_exc[rr]
                                         : sp.region_offsets[rr + 1] - a;
        if (pool <= 0) continue;
        src = a + (int32_t)g.below((uint32_t)pool);
        size_t h = ((uint64_t)src * 0x9E3779B97F4A7C15ull) >> 20;
        bool dup = false;
        for (;;) {
          h &= hmask;
          if (hset[h] == -1) break;
          if (hset[h] == src) { dup = true; break; }
          ++h;
        }
        if (dup) continue;
        hset[h] = src;
        used.push_back(h);
        break;
      }
      emit(src, tgt, false);
    }
    for (size_t h : used) hset[h] = -1;
  }

  // delay and BF16 weight of the edge src -> tgt, from a stream keyed by the pair
  void attributes(int32_t src, int32_t tgt, bool within, uint8_t* d, uint16_t* w) const {
    Rng g(sp.seed, 0xED6Eull ^ ((uint64_t)(uint32_t)src << 20), (uint64_t)tgt);
    int32_t lo = within ? sp.d_within_min : sp.d_cross_min;
    int32_t hi = within ? sp.d_within_max : sp.d_cross_max;
    *d = (uint8_t)(lo + (int32_t)g.below((uint32_t)(hi - lo + 1)));
    *w = f32_to_bf16_rne((float)std::exp(sp.w_mu + sp.w_sigma * g.normal()));
  }
};

}  // namespace

extern "C" {

// Fill a CSR by source with rows sorted by (delay, target).  The caller
// allocates row_ptr[N+1] and col/w_bf16/delay[N*k_in].
// Returns 0, or a negative code for an unusable spec.
int synth_graph(const SynthSpec* spp, int64_t* row_ptr, int32_t* col,
                uint16_t* w_bf16, uint8_t* delay, int32_t nthreads) {
  if (!spp || !row_ptr || !col || !w_bf16 || !delay) return -1;
  const SynthSpec& sp = *spp;
  const int32_t N = sp.n_neurons, R = sp.n_regions;
  if (N <= 1 || R <= 0 || sp.region_offsets[0] != 0 || sp.region_offsets[R] != N) return -2;
  if (sp.k_in <= 0 || sp.k_within < 0 || sp.k_within > sp.k_in) return -3;
  for (int32_t r = 0; r < R; ++r) {
    int32_t nr = sp.region_offsets[r + 1] - sp.region_offsets[r];
    int32_t kw = R == 1 ? sp.k_in : sp.k_within;
    if (nr <= 0 || kw > nr - 1) return -4;
    if (sp.n_exc[r] < 0 || sp.n_exc[r] > nr) return -5;
  }
  if (sp.d_within_min < 1 || sp.d_within_max < sp.d_within_min || sp.d_within_max > 255)
    return -6;
  if (R > 1 && (sp.d_cross_min < 1 || sp.d_cross_max < sp.d_cross_min || sp.d_cross_max > 255))
    return -6;
  // cumulative source-region distributions
  std::vector<std::vector<double>> cdf((size_t)R);
  for (int32_t r = 0; r < R && R > 1; ++r) {
    cdf[(size_t)r].resize((size_t)R);
    double acc = 0.0, tot = 0.0;
    for (int32_t c = 0; c < R; ++c) {
      double v = c == r ? 0.0 : (sp.region_prob ? sp.region_prob[(int64_t)r * R + c] : 1.0);
      if (sp.cross_exc_only && sp.n_exc[c] == 0) v = 0.0;
      tot += v;
    }
    if (tot <= 0.0) return -7;
    for (int32_t c = 0; c < R; ++c) {
      double v = c == r ? 0.0 : (sp.region_prob ? sp.region_prob[(int64_t)r * R + c] : 1.0);
      if (sp.cross_exc_only && sp.n_exc[c] == 0) v = 0.0;
      acc += v / tot;
      cdf[(size_t)r][(size_t)c] = acc;
    }
    cdf[(size_t)r][(size_t)R - 1] = 1.0;
  }
  std::vector<int32_t> region_of((size_t)N);
  for (int32_t r = 0; r < R; ++r)
    for (int32_t i = sp.region_offsets[r]; i < sp.region_offsets[r + 1]; ++i)
      region_of[(size_t)i] = r;

#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  // pass 1: out-degrees
  std::vector<std::atomic<int32_t>> outdeg((size_t)N);
  for (auto& x : outdeg) x.store(0, std::memory_order_relaxed);
#pragma omp parallel
  {
    TargetSampler ts(sp, cdf);
#pragma omp for schedule(dynamic, 256)
    for (int32_t i = 0; i < N; ++i)
      ts.run(i, region_of[(size_t)i], [&](int32_t s, int32_t, bool) {
        outdeg[(size_t)s].fetch_add(1, std::memory_order_relaxed);
      });
  }
  row_ptr[0] = 0;
  for (int32_t j = 0; j < N; ++j) row_ptr[j + 1] = row_ptr[j] + outdeg[(size_t)j].load();
  const int64_t E = row_ptr[N];
  // pass 2: the same draws again, scattered into the output rows (in
  // arrival order); no memory beyond the output itself
  for (auto& x : outdeg) x.store(0, std::memory_order_relaxed);
#pragma omp parallel
  {
    TargetSampler ts(sp, cdf);
#pragma omp for schedule(dynamic, 256)
    for (int32_t i = 0; i < N; ++i)
      ts.run(i, region_of[(size_t)i], [&](int32_t s, int32_t t, bool within) {
        uint8_t d;
        uint16_t w;
        ts.attributes(s, t, within, &d, &w);
        const int64_t e = row_ptr[s] + outdeg[(size_t)s].fetch_add(1, std::memory_order_relaxed);
        col[e] = i;
        w_bf16[e] = w;
        delay[e] = d;
      });
  }
  // pass 3: sort each row by (delay, target) through a per-thread buffer of
  // packed keys (one row at a time)
#pragma omp parallel
  {
    std::vector<uint64_t> key;
#pragma omp for schedule(dynamic, 1024)
    for (int32_t j = 0; j < N; ++j) {
      const int64_t a = row_ptr[j], n = row_ptr[j + 1] - a;
      key.resize((size_t)n);
      for (int64_t p = 0; p < n; ++p)
        key[(size_t)p] = ((uint64_t)delay[a + p] << 56) | ((uint64_t)(uint32_t)col[a + p] << 16) |
                         (uint64_t)w_bf16[a + p];
      std::sort(key.begin(), key.end());
      for (int64_t p = 0; p < n; ++p) {
        const uint64_t k = key[(size_t)p];
        delay[a + p] = (uint8_t)(k >> 56);
        col[a + p] = (int32_t)((k >> 16) & 0xFFFFFFFFull);
        w_bf16[a + p] = (uint16_t)(k & 0xFFFFull);
      }
    }
  }
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Cortical micro-column networks (Extended Data Table 3; Supplementary
// Sec. 2, Eqs. 5-6): every region (voxel) holds the same list of
// populations; a neuron of population i receives exactly k_local[i][j]
// synapses from population j of its own voxel (sources uniform without
// replacement, no autapse) and k_cc[i] cortico-cortical synapses from
// excitatory neurons of other voxels, the source voxel following the
// row-stochastic region matrix (no multapse).
extern "C" {

struct ColumnSpec {
  int32_t n_voxels, n_pops;
  const int32_t* pop_offset;  // [n_pops + 1] offsets of the populations inside a voxel
  int32_t voxel_size;         // neurons per voxel (= pop_offset[n_pops])
  int32_t n_exc;              // excitatory neurons per voxel (populations come E first)
  const int32_t* k_local;     // [n_pops][n_pops]
  const int32_t* k_cc;        // [n_pops]
  const double* region_prob;  // [V*V] row-stochastic, diagonal ignored
  int32_t d_within_min, d_within_max, d_cross_min, d_cross_max;
  double w_mu, w_sigma;
  uint64_t seed;
};

}  // extern "C"

namespace {

struct ColumnSampler {
  const ColumnSpec& sp;
  const std::vector<std::vector<double>>& cdf;
  std::vector<uint64_t> bitmap;
  std::vector<int32_t> chosen, hset;
  std::vector<size_t> used;

  ColumnSampler(const ColumnSpec& s, const std::vector<std::vector<double>>& c) : sp(s), cdf(c) {
    int32_t maxp = 1, maxcc = 1;
    for (int32_t p = 0; p < s.n_pops; ++p) {
      maxp = std::max(maxp, s.pop_offset[p + 1] - s.pop_offset[p]);
      maxcc = std::max(maxcc, s.k_cc[p]);
    }
    bitmap.assign((size_t)maxp / 64 + 1, 0ull);
    int hs = 16;
    while (hs < 4 * (maxcc + 1)) hs <<= 1;
    hset.assign((size_t)hs, -1);
  }

  template <class F>
  void run(int32_t tgt, F&& emit) {
    Rng g(sp.seed, 0xC01Full, (uint64_t)tgt);
    const int32_t v = tgt / sp.voxel_size, local = tgt % sp.voxel_size;
    int32_t pi = 0;
    while (local >= sp.pop_offset[pi + 1]) ++pi;
    const int32_t vbase = v * sp.voxel_size;
    for (int32_t pj = 0; pj < sp.n_pops; ++pj) {
      const int32_t a = sp.pop_offset[pj], n = sp.pop_offset[pj + 1] - a;
      const bool same = pj == pi;
      const int32_t m = n - (same ? 1 : 0);  // candidates (self excluded)
      const int32_t k = std::min(sp.k_local[pi * sp.n_pops + pj], m);
      if (k <= 0) continue;
      const int32_t self = local - a;
      chosen.clear();
      for (int32_t j = m - k; j < m; ++j) {  // Floyd's sampling
        int32_t t = (int32_t)g.below((uint32_t)j + 1);
        int32_t pick = (bitmap[t >> 6] >> (t & 63)) & 1ull ? j : t;
        bitmap[pick >> 6] |= 1ull << (pick & 63);
        chosen.push_back(pick);
      }
      for (int32_t c : chosen) {
        bitmap[c >> 6] &= ~(1ull << (c & 63));
        const int32_t idx = same && c >= self ? c + 1 : c;
        emit(vbase + a + idx, tgt, true);
      }
    }
    const int32_t kc = sp.n_voxels > 1 ? sp.k_cc[pi] : 0;
    if (kc <= 0 || sp.n_exc <= 0) return;
    const size_t hmask = hset.size() - 1;
    used.clear();
    for (int32_t q = 0; q < kc; ++q) {
      int32_t src;
      for (;;) {
        const std::vector<double>& row = cdf[(size_t)v];
        int32_t vv = (int32_t)(std::lower_bound(row.begin(), row.end(), g.unit()) - row.begin());
        if (vv >= sp.n_voxels) vv = sp.n_voxels - 1;
        if (vv == v) continue;
        src = vv * sp.voxel_size + (int32_t)g.below((uint32_t)sp.n_exc);
        size_t h = ((uint64_t)src * 0x9E3779B97F4A7C15ull) >> 20;
        bool dup = false;
        for (;;) {
          h &= hmask;
          if (hset[h] == -1) break;
          if (hset[h] == src) { dup = true; break; }
          ++h;
        }
        if (dup) continue;
        hset[h] = src;
        used.push_back(h);
        break;
      }
      emit(src, tgt, false);
    }
    for (size_t h : used) hset[h] = -1;
  }

  void attributes(int32_t src, int32_t tgt, bool within, uint8_t* d, uint16_t* w) const {
    Rng g(sp.seed, 0xED6Eull ^ ((uint64_t)(uint32_t)src << 20), (uint64_t)tgt);
    int32_t lo = within ? sp.d_within_min : sp.d_cross_min;
    int32_t hi = within ? sp.d_within_max : sp.d_cross_max;
    *d = (uint8_t)(lo + (int32_t)g.below((uint32_t)(hi - lo + 1)));
    *w = f32_to_bf16_rne((float)std::exp(sp.w_mu + sp.w_sigma * g.normal()));
  }
};

}  // namespace

extern "C" {

// Out-degrees first (row_ptr), then the CSR by source sorted by (delay,
// target), as synth_graph.  Returns 0 or a negative code.
int synth_columns(const ColumnSpec* spp, int64_t* row_ptr, int32_t* col, uint16_t* w_bf16,
                  uint8_t* delay, int32_t nthreads) {
  if (!spp || !row_ptr) return -1;
  const ColumnSpec& sp = *spp;
  const int32_t V = sp.n_voxels, P = sp.n_pops;
  if (V < 1 || P < 1 || sp.voxel_size < 2 || sp.pop_offset[0] != 0 ||
      sp.pop_offset[P] != sp.voxel_size || sp.n_exc < 0 || sp.n_exc > sp.voxel_size)
    return -2;
  if ((int64_t)V * sp.voxel_size >= (int64_t(1) << 31)) return -3;
  if (sp.d_within_min < 1 || sp.d_within_max < sp.d_within_min || sp.d_within_max > 255 ||
      sp.d_cross_min < 1 || sp.d_cross_max < sp.d_cross_min || sp.d_cross_max > 255)
    return -6;
  std::vector<std::vector<double>> cdf((size_t)V);
  for (int32_t r = 0; r < V && V > 1; ++r) {
    cdf[(size_t)r].resize((size_t)V);
    double acc = 0.0, tot = 0.0;
    for (int32_t c = 0; c < V; ++c) tot += c == r ? 0.0 : (sp.region_prob ? sp.region_prob[(int64_t)r * V + c] : 1.0);
    if (tot <= 0.0) return -7;
    for (int32_t c = 0; c < V; ++c) {
      acc += (c == r ? 0.0 : (sp.region_prob ? sp.region_prob[(int64_t)r * V + c] : 1.0)) / tot;
      cdf[(size_t)r][(size_t)c] = acc;
    }
    cdf[(size_t)r][(size_t)V - 1] = 1.0;
  }
  const int32_t N = V * sp.voxel_size;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  std::vector<std::atomic<int32_t>> outdeg((size_t)N);
  for (auto& x : outdeg) x.store(0, std::memory_order_relaxed);
#pragma omp parallel
  {
    ColumnSampler cs(sp, cdf);
#pragma omp for schedule(dynamic, 256)
    for (int32_t i = 0; i < N; ++i)
      cs.run(i, [&](int32_t s, int32_t, bool) { outdeg[(size_t)s].fetch_add(1, std::memory_order_relaxed); });
  }
  row_ptr[0] = 0;
  for (int32_t j = 0; j < N; ++j) row_ptr[j + 1] = row_ptr[j] + outdeg[(size_t)j].load();
  if (!col) return 0;  // out-degrees only: the caller sizes the edge arrays
  const int64_t E = row_ptr[N];
  std::vector<uint64_t> key((size_t)E);
  for (auto& x : outdeg) x.store(0, std::memory_order_relaxed);
#pragma omp parallel
  {
    ColumnSampler cs(sp, cdf);
#pragma omp for schedule(dynamic, 256)
    for (int32_t i = 0; i < N; ++i)
      cs.run(i, [&](int32_t s, int32_t t, bool within) {
        uint8_t d;
        uint16_t w;
        cs.attributes(s, t, within, &d, &w);
        int32_t p = outdeg[(size_t)s].fetch_add(1, std::memory_order_relaxed);
        key[(size_t)(row_ptr[s] + p)] = ((uint64_t)d << 56) | ((uint64_t)(uint32_t)i << 16) | (uint64_t)w;
      });
  }
#pragma omp parallel for schedule(dynamic, 1024)
  for (int32_t j = 0; j < N; ++j) {
    uint64_t* a = key.data() + row_ptr[j];
    uint64_t* b = key.data() + row_ptr[j + 1];
    std::sort(a, b);
    for (int64_t e = row_ptr[j]; e < row_ptr[j + 1]; ++e) {
      uint64_t k = key[(size_t)e];
      delay[e] = (uint8_t)(k >> 56);
      col[e] = (int32_t)((k >> 16) & 0xFFFFFFFFull);
      w_bf16[e] = (uint16_t)(k & 0xFFFFull);
    }
  }
  return 0;
}

}  // extern "C"

// Host engine and the dbnet_* C ABI (see include/dbnet.h).
//
// Create: host-side checks that cost O(N + R), then the edge arrays are
// copied to the device in chunks of rows, each chunk validated by one
// warp-per-row kernel (target range, delay range and order, weights -> BF16,
// in-degrees, largest weight) that writes the interleaved edge records (6
// bytes, or 8 with a second weight) and the per-delay segment table of its
// rows; the fixed-point scale is chosen from those, the region constants are
// derived in FP64 and rounded to FP32 once, and the initial state is drawn
// on the device.  A graph with two weights per edge makes the engine keep
// four accumulator channels per neuron.
//
// Step: (deliver, update) kernel pairs on the handle's stream, replayed from
// a captured CUDA graph of kChunk steps; all per-step indices live in device
// memory, so the same graph serves every chunk.
#include <cuda_runtime.h>
#include <omp.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dbnet.h"
#include "engine.h"
#include "host.h"

namespace dbn {

thread_local std::string g_last_error;
thread_local Arena* g_arena = nullptr;
thread_local void* g_alloc_stream = nullptr;

namespace {
std::mutex g_hook_mu;
AllocHook g_hook;
}  // namespace

AllocHook current_alloc_hook() {
  std::lock_guard<std::mutex> lock(g_hook_mu);
  return g_hook;
}

// ---------------------------------------------------------------- graph ----
// The largest byte of a[0..n): over the host's cores for large arrays (the
// delays of a 2e10-edge graph are 20 GB).
static unsigned max_byte(const uint8_t* a, int64_t n) {
  constexpr int64_t kPer = int64_t(1) << 26;  // at least 64 MB per thread
  const int64_t want = (n + kPer - 1) / kPer;
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = (int)std::min<int64_t>(std::min(hw, 64), std::max<int64_t>(want, 1));
  auto span_max = [a](int64_t b, int64_t e) {
    unsigned m = 0;
    for (int64_t i = b; i < e; ++i) m = std::max<unsigned>(m, a[i]);
    return m;
  };
  if (nt <= 1) return span_max(0, n);
  std::vector<unsigned> part((size_t)nt, 0u);
  std::vector<std::thread> th;
  const int64_t per = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] { part[(size_t)t] = span_max(std::min(n, t * per), std::min(n, (t + 1) * per)); });
  for (auto& x : th) x.join();
  return *std::max_element(part.begin(), part.end());
}

// Host-to-device copies from pageable host memory through pinned slices:
// the host's cores copy each slice into pinned memory while the DMA of the
// previous slices runs (CUDA's own path for pageable sources copies
// on one thread); pinned sources are copied directly.
class HostStager {
 public:
  static constexpr size_t kSlice = size_t(64) << 20;
  static constexpr int kSlices = 4;
  explicit HostStager(cudaStream_t s) : s_(s) {}
  HostStager(const HostStager&) = delete;
  HostStager& operator=(const HostStager&) = delete;
  ~HostStager() {
    for (int i = 0; i < kSlices; ++i) {
      if (ev_[i]) {
        cudaEventSynchronize(ev_[i]);  // its copy has left the slice
        cudaEventDestroy(ev_[i]);
      }
      if (buf_[i]) cudaFreeHost(buf_[i]);
    }
  }
  void copy(void* dst, const void* src, size_t n) {
    if (n == 0) return;
    cudaPointerAttributes at{};
    const bool pinned = cudaPointerGetAttributes(&at, src) == cudaSuccess && at.type == cudaMemoryTypeHost;
    cudaGetLastError();  // clear a lookup failure on an unregistered pointer
    if (pinned || n < kSlice) {
      CK(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s_));
      return;
    }
    if (!buf_[0]) {
      for (int i = 0; i < kSlices; ++i) {
        CK(cudaHostAlloc(&buf_[i], kSlice, cudaHostAllocDefault));
        CK(cudaEventCreateWithFlags(&ev_[i], cudaEventDisableTiming));
      }
    }
    const auto* from = static_cast<const unsigned char*>(src);
    auto* to = static_cast<unsigned char*>(dst);
    for (size_t o = 0; o < n; o += kSlice) {
      const size_t m = std::min(kSlice, n - o);
      const int b = next_;
      next_ = (next_ + 1) % kSlices;
      CK(cudaEventSynchronize(ev_[b]));  // the slice's previous copy is done
      fill(static_cast<unsigned char*>(buf_[b]), from + o, m);
      CK(cudaMemcpyAsync(to + o, buf_[b], m, cudaMemcpyHostToDevice, s_));
      CK(cudaEventRecord(ev_[b], s_));
    }
  }

 private:
  static void fill(unsigned char* dst, const unsigned char* src, size_t m) {
    const int nt = std::max(1, std::min(omp_get_num_procs(), 16));
    const size_t per = ((m + nt - 1) / nt + 4095) & ~size_t(4095);
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int t = 0; t < nt; ++t) {
      const size_t lo = std::min(m, (size_t)t * per), hi = std::min(m, lo + per);
      if (hi > lo) std::memcpy(dst + lo, src + lo, hi - lo);
    }
  }
  cudaStream_t s_;
  void* buf_[kSlices] = {};
  cudaEvent_t ev_[kSlices] = {};
  int next_ = 0;
};

std::shared_ptr<GraphDev> upload_graph(const dbnet_graph_t* g, cudaStream_t s) {
  if (!g) raise(DBNET_EINVAL, "graph is NULL");
  const int32_t N = g->n_neurons, R = g->n_regions;
  if (N < 1 || R < 1) raise(DBNET_EINVAL, "n_neurons and n_regions must be >= 1");
  if (!g->region_offsets || !g->n_exc || !g->row_ptr) raise(DBNET_EINVAL, "NULL graph array");
  if (g->weight_dtype != DBNET_WEIGHT_F32 && g->weight_dtype != DBNET_WEIGHT_BF16)
    raise(DBNET_EINVAL, "weight_dtype must be DBNET_WEIGHT_F32 or DBNET_WEIGHT_BF16");
  if (g->region_offsets[0] != 0 || g->region_offsets[R] != N)
    raise(DBNET_EINVAL, "region_offsets must start at 0 and end at n_neurons");
  for (int32_t r = 0; r < R; ++r) {
    const int32_t sz = g->region_offsets[r + 1] - g->region_offsets[r];
    if (sz < 1) raise(DBNET_EINVAL, "region_offsets must be strictly increasing");
    if (g->n_exc[r] < 0 || g->n_exc[r] > sz) raise(DBNET_EINVAL, "n_exc out of range");
  }
  if (g->row_ptr[0] != 0) raise(DBNET_EINVAL, "row_ptr[0] must be 0");
  for (int32_t j = 0; j < N; ++j)
    if (g->row_ptr[j + 1] < g->row_ptr[j]) raise(DBNET_EINVAL, "row_ptr must be non-decreasing");
  const int64_t E = g->row_ptr[N];
  if (E >= (int64_t(1) << 47)) raise(DBNET_EINVAL, "too many edges");
  if (E > 0 && (!g->col || !g->weight || !g->delay)) raise(DBNET_EINVAL, "NULL edge array");

  auto gd = std::make_shared<GraphDev>();
  gd->N = N;
  gd->R = R;
  gd->E = E;
  gd->ro_h.assign(g->region_offsets, g->region_offsets + R + 1);
  gd->nexc_h.assign(g->n_exc, g->n_exc + R);
  // the largest delay and row length fix the segment table's shape
  const unsigned dmax_h = E > 0 ? max_byte(g->delay, E) : 0u;
  gd->max_delay = (int32_t)std::max(1u, dmax_h);
  int64_t max_out = 0;
  for (int32_t j = 0; j < N; ++j) max_out = std::max(max_out, g->row_ptr[j + 1] - g->row_ptr[j]);
  gd->seg_kind = max_out < 65536 ? kSeg16 : kSeg32;  // u16 counts when every row is short
  // edges per row and delay on a sample of rows: the delays from which all
  // segments are short enough to hand on at emission
  {
    const int32_t every = std::max<int32_t>(1, N / 65536);
    std::vector<double> per_delay(256, 0.0);
    int64_t rows = 0;
    for (int32_t j = 0; j < N; j += every, ++rows)
      for (int64_t e = g->row_ptr[j]; e < g->row_ptr[j + 1]; ++e) per_delay[g->delay[e]] += 1.0;
    int32_t from = 0;
    for (int32_t d = gd->max_delay; d >= 1 && rows > 0; --d) {
      if (per_delay[(size_t)d] / (double)rows >= kEmitSegEdges) break;
      from = d;
    }
    gd->emit_from = E > 0 ? from : 0;
  }
  const int32_t per16 = gd->seg_kind == kSeg16 ? 8 : 4;  // entries per 16 bytes
  gd->seg_stride = (gd->max_delay + per16 - 1) / per16 * per16;
  const int64_t seg_bytes = (int64_t)N * gd->seg_stride * (gd->seg_kind == kSeg16 ? 2 : 4);

  gd->row_ptr.alloc(N + 1);
  gd->ro.alloc(R + 1);
  gd->two_w = g->weight2 != nullptr;
  gd->rec.alloc((gd->two_w ? 4 : 3) * E + 4);  // 8 bytes of padding: the delivery reads whole words
  gd->seg.alloc(seg_bytes);
  CK(cudaMemcpyAsync(gd->row_ptr.p, g->row_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(gd->ro.p, g->region_offsets, sizeof(int32_t) * (R + 1), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(gd->seg.p, 0, (size_t)seg_bytes, s));
  DevBuf<int32_t> indeg;
  indeg.alloc(N);
  DevBuf<unsigned> scal;  // wmax bits, unused, err, kin_max
  scal.alloc(4);
  CK(cudaMemsetAsync(indeg.p, 0, sizeof(int32_t) * N, s));
  CK(cudaMemsetAsync(scal.p, 0, sizeof(unsigned) * 4, s));
  // rows in chunks of about kIngestEdges edges through staging buffers, so
  // the device never holds more than the records and one chunk
  if (E > 0) {
    constexpr int64_t kIngestEdges = int64_t(1) << 27;
    const int64_t cap = std::min(E, std::max(kIngestEdges, max_out));
    const int64_t wsz = g->weight_dtype == DBNET_WEIGHT_BF16 ? 2 : 4;
    DevBuf<int32_t> col_st;
    DevBuf<uint8_t> w_st, w2_st, d_st;
    col_st.alloc(cap);
    w_st.alloc(cap * wsz);
    if (gd->two_w) w2_st.alloc(cap * wsz);
    d_st.alloc(cap);
    HostStager stage(s);
    int32_t j0 = 0;
    while (j0 < N) {
      int32_t j1 = j0 + 1;
      while (j1 < N && g->row_ptr[j1 + 1] - g->row_ptr[j0] <= cap) ++j1;
      const int64_t e0 = g->row_ptr[j0], ne = g->row_ptr[j1] - e0;
      if (ne > 0) {
        stage.copy(col_st.p, g->col + e0, sizeof(int32_t) * ne);
        stage.copy(d_st.p, g->delay + e0, ne);
        stage.copy(w_st.p, static_cast<const uint8_t*>(g->weight) + e0 * wsz, ne * wsz);
        if (gd->two_w) stage.copy(w2_st.p, static_cast<const uint8_t*>(g->weight2) + e0 * wsz, ne * wsz);
        launch_ingest(N, j0, j1, e0, gd->row_ptr.p, col_st.p, w_st.p,
                      gd->two_w ? w2_st.p : nullptr, g->weight_dtype, d_st.p,
                      gd->rec.p, gd->max_delay, gd->seg_stride, gd->seg.p, gd->seg_kind, indeg.p,
                      scal.p + 0, scal.p + 2, s);
        CK(cudaGetLastError());
      }
      j0 = j1;
    }
    CK(cudaStreamSynchronize(s));  // the staging buffers are freed next
  }
  launch_max_reduce(indeg.p, N, scal.p + 3, s);
  CK(cudaGetLastError());
  unsigned h[4];
  CK(cudaMemcpyAsync(h, scal.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const unsigned err = h[2];
  if (err & kErrTarget) raise(DBNET_EINVAL, "an edge target is outside [0, n_neurons)");
  if (err & kErrDelayRange) raise(DBNET_EINVAL, "an edge delay is 0 (delays are 1..255 steps)");
  if (err & kErrDelayOrder) raise(DBNET_EINVAL, "delays must be non-decreasing within each row");
  if (err & kErrWeight) raise(DBNET_EINVAL, "weights must be finite and non-negative");
  gd->rounded = (err & kErrRounded) != 0;
  float wmax;
  std::memcpy(&wmax, &h[0], 4);
  gd->w_max = (double)wmax;
  gd->kin_max = (int32_t)h[3];
  return gd;
}

// ---------------------------------------------------- region constants ----
static bool finite(double x) { return std::isfinite(x); }

int32_t bin_lead(const dbnet_options_t& o) {
  return o.bin_spikes ? (int32_t)std::lrint(o.bin_ms / o.dt_ms) - 1 : 0;
}

void check_params(const dbnet_region_params_t& p, double dt, int32_t min_ref) {
  if (!(p.C > 0) || !finite(p.C)) raise(DBNET_EINVAL, "C must be > 0");
  if (std::lrint(p.Tref / dt) < min_ref)
    raise(DBNET_EINVAL, "with spike binning T_ref must be at least one bin minus one step");
  if (!(p.gL >= 0) || !finite(p.gL)) raise(DBNET_EINVAL, "gL must be >= 0");
  for (double v : {p.VL, p.Vth, p.Vreset, p.I_ext})
    if (!finite(v)) raise(DBNET_EINVAL, "non-finite membrane constant");
  if (!(p.Tref >= 0) || std::lrint(p.Tref / dt) > 255) raise(DBNET_EINVAL, "Tref must be in [0, 255 dt]");
  for (int u = 0; u < 4; ++u) {
    if (!(p.tau_u[u] > 0)) raise(DBNET_EINVAL, "tau_u must be > 0");
    if (!finite(p.g_u[u]) || !finite(p.Vu[u])) raise(DBNET_EINVAL, "non-finite synapse constant");
  }
  if (!(p.drive_rate_hz >= 0) || !(p.drive_K >= 0) || !(p.w_ext >= 0) || !finite(p.w_ext) ||
      !finite(p.drive_rate_hz * p.drive_K))
    raise(DBNET_EINVAL, "drive constants must be finite and >= 0");
  if (!finite(p.ou_mu) || !(p.ou_sigma >= 0) || !finite(p.ou_sigma))
    raise(DBNET_EINVAL, "ou_mu must be finite and ou_sigma finite and >= 0");
  if ((p.ou_mu != 0.0 || p.ou_sigma != 0.0) && !(p.ou_tau > 0 && finite(p.ou_tau)))
    raise(DBNET_EINVAL, "ou_tau must be > 0 when the OU current is on");
  if (!(p.iext_shape >= 0) || !finite(p.iext_shape))
    raise(DBNET_EINVAL, "iext_shape must be finite and >= 0");
}

static bool ou_on(const dbnet_region_params_t& p) { return p.ou_mu != 0.0 || p.ou_sigma != 0.0; }
static int32_t ext_bits(const dbnet_region_params_t& p) {
  return (ou_on(p) ? kExtOU : 0) | (p.iext_shape > 0.0 ? kExtHet : 0);
}

// Per-neuron injected-current factor G / k, G ~ Gamma(k, 1), for local
// neuron i: the Marsaglia-Tsang method (ACM TOMS 26(3), 2000) on the
// neuron's Philox words of stream 5 -- attempt a uses counter (0, i, 5, a):
// word 0 gives a Box-Muller normal, word 1 the acceptance uniform, word 2
// (k < 1) the uniform of G(k) = G(k + 1) U^(1/k) -- in FP64.
static double unit_open(unsigned long long w) { return ((double)(w >> 32) + 1.0) * std::ldexp(1.0, -32); }
static double normal_of(unsigned long long w) {
  const double u1 = unit_open(w);
  const double u2 = (double)(w & 0xFFFFFFFFull) * std::ldexp(1.0, -32);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * 3.14159265358979323846 * u2);
}
static double gamma_of(double k, unsigned long long seed, unsigned long long net_id, int64_t i) {
  const double kk = k < 1.0 ? k + 1.0 : k;
  const double d = kk - 1.0 / 3.0;
  const double c = 1.0 / std::sqrt(9.0 * d);
  for (unsigned long long a = 0;; ++a) {
    unsigned long long w[4] = {0ull, (unsigned long long)i, 5ull, a};
    philox4x64_10(w, seed, net_id);
    const double x = normal_of(w[0]);
    const double t = 1.0 + c * x;
    if (t <= 0.0) continue;
    const double v = t * t * t;
    const double u = unit_open(w[1]);
    if (std::log(u) < 0.5 * x * x + d - d * v + d * std::log(v)) {
      double gm = d * v;
      if (k < 1.0) gm = gm * std::pow(unit_open(w[2]), 1.0 / k);
      return gm;
    }
  }
}

// Thresholds of the integer-inversion Poisson draw: floor(P(X <= k) 2^32) for
// the leading k (at most 16) whose value stays below 2^32.
int poisson_thresholds(double lam, uint32_t* thr) {
  double p = std::exp(-lam);
  double cdf = p;
  int n = 0;
  for (int k = 0; k < kMaxThr; ++k) {
    const double t = std::floor(std::ldexp(cdf, 32));
    if (t >= 4294967296.0) break;
    thr[k] = (uint32_t)t;
    n = k + 1;
    p = p * lam;
    p = p / (double)(k + 1);
    cdf = cdf + p;
  }
  return n;
}

RegionConst region_const(const dbnet_region_params_t& p, double dt, int S, int32_t start,
                         int32_t end, int32_t exc_end) {
  RegionConst c;
  std::memset(&c, 0, sizeof(c));
  c.dtC = (float)(dt / p.C);
  c.gL = (float)p.gL;
  c.VL = (float)p.VL;
  c.Vth = (float)p.Vth;
  c.Vreset = (float)p.Vreset;
  c.Iext = (float)p.I_ext;
  for (int u = 0; u < 4; ++u) {
    c.g[u] = (float)p.g_u[u];
    c.Vu[u] = (float)p.Vu[u];
    c.dec[u] = (float)std::exp(-dt / p.tau_u[u]);
  }
  c.n_ref = (int32_t)std::lrint(p.Tref / dt);
  c.q_ext = (int32_t)std::lrint(std::ldexp(p.w_ext, S));
  c.n_thr = poisson_thresholds(p.drive_K * p.drive_rate_hz * dt * 1e-3, c.thr);
  c.start = start;
  c.end = end;
  c.exc_end = exc_end;
  c.ext = ext_bits(p);
  if (ou_on(p)) {
    c.ou_mu = (float)p.ou_mu;
    c.ou_k = (float)(dt / p.ou_tau);
    c.ou_s = (float)(p.ou_sigma * std::sqrt(2.0 * dt / p.ou_tau));
  }
  return c;
}

int choose_shift(const GraphDev& g, double wext_max, int32_t requested) {
  auto bound = [&](int S) {
    return (double)g.kin_max * std::rint(std::ldexp(g.w_max, S)) +
           16.0 * std::rint(std::ldexp(wext_max, S));
  };
  if (requested < 0 || requested > 30) raise(DBNET_EINVAL, "fixed_shift must be in 0..30");
  int S = requested > 0 ? requested : 16;
  if (requested == 0)
    while (S > 0 && bound(S) > 2147483647.0) --S;
  if (bound(S) > 2147483647.0)
    raise(DBNET_EOVERFLOW, "one step's worst-case arrivals overflow int32 at this fixed_shift");
  return S;
}

void check_options(const dbnet_options_t& o) {
  if (!(o.dt_ms > 0) || !finite(o.dt_ms)) raise(DBNET_EINVAL, "dt_ms must be > 0");
  const double spb = o.bin_ms / o.dt_ms;
  if (!(spb >= 0.5) || std::fabs(spb - std::rint(spb)) > 1e-6 * spb)
    raise(DBNET_EINVAL, "bin_ms must be a whole number of steps");
  const double bpt = o.tr_ms / o.bin_ms;
  if (!(bpt >= 0.5) || std::fabs(bpt - std::rint(bpt)) > 1e-6 * bpt)
    raise(DBNET_EINVAL, "tr_ms must be a whole number of bins");
  if (o.precision != 32) raise(DBNET_EUNSUPPORTED, "the device path computes FP32 state (precision 32)");
  if (o.raster_capacity < 0 || o.bold_capacity < 0) raise(DBNET_EINVAL, "negative capacity");
  if (!(o.bw_alpha > 0) || !(o.bw_tau > 0) || !(o.bw_rho > 0 && o.bw_rho < 1))
    raise(DBNET_EINVAL, "Balloon-Windkessel constants out of range");
  if (!finite(o.z_scale)) raise(DBNET_EINVAL, "z_scale must be finite");
  if (o.fixed_shift < 0 || o.fixed_shift > 30) raise(DBNET_EINVAL, "fixed_shift must be in 0..30");
  if (o.autotune_at < -1) raise(DBNET_EINVAL, "autotune_at must be -1 or a step index");
  if (o.bin_spikes != 0 && o.bin_spikes != 1) raise(DBNET_EINVAL, "bin_spikes must be 0 or 1");
  if (o.emit_delay < -1 || o.emit_delay > 255) raise(DBNET_EINVAL, "emit_delay must be -1..255");
  if (o.schedule < DBNET_SCHEDULE_AUTO || o.schedule > DBNET_SCHEDULE_PERSISTENT)
    raise(DBNET_EINVAL, "schedule must be one of DBNET_SCHEDULE_*");
  if (o.deliver_blocks < 0 || o.deliver_blocks == 1 || o.deliver_blocks > (1 << 20))
    raise(DBNET_EINVAL, "deliver_blocks must be 0 (automatic) or 2 .. 2^20");
}

// --------------------------------------------------------------- engine ----
void Engine::init(const std::vector<InstSpec>& specs, void* user_stream) {
  const int n = (int)specs.size();
  // fixed-point scale shared by the engine
  double wext_max = 0.0;
  for (const auto& sp : specs)
    for (const auto& p : sp.params) wext_max = std::max(wext_max, p.w_ext);
  int S = 16;
  for (int k = 0; k < n; ++k) S = std::min(S, choose_shift(*specs[k].graph, wext_max, specs[0].opt.fixed_shift));
  shift_S = S;
  // layout: instances end to end, each on whole tiles
  int64_t tiles = 0;
  int32_t regions = 0, dmax_all = 1;
  for (const auto& sp : specs) {
    tiles += (sp.graph->N + kTile - 1) / kTile;
    regions += sp.graph->R;
    dmax_all = std::max(dmax_all, sp.graph->max_delay);
  }
  bool any_ext = false, four = false;
  for (const auto& sp : specs) {
    for (const auto& p : sp.params) any_ext = any_ext || ext_bits(p) != 0;
    four = four || sp.graph->two_w;
  }
  // delays handed on at emission: the option, or (0) the graphs' own
  // threshold (instances share one graph in an ensemble)
  int32_t emit_from = 0;
  const int32_t want = specs[0].opt.emit_delay;
  if (want > 0) {
    emit_from = want;
  } else if (want == 0) {
    emit_from = specs[0].graph->emit_from;
    for (const auto& sp : specs)
      if (sp.graph->emit_from != emit_from) emit_from = 0;
  }
  // with spike binning a spike waits up to spb - 1 steps for its bin to end
  init_pool(n, tiles, regions, dmax_all + 1 + bin_lead(specs[0].opt), specs[0].opt, user_stream,
            any_ext, four, emit_from > dmax_all ? 0 : emit_from);
  int64_t t = 0;
  int32_t r = 0;
  for (int k = 0; k < n; ++k) {
    place(k, specs[k], (int32_t)t, r, S, LLONG_MAX);
    t += (specs[k].graph->N + kTile - 1) / kTile;
    r += specs[k].graph->R;
  }
  set_extent((int32_t)tiles, regions);
  CK(cudaStreamSynchronize(stream));
}

void Engine::init_pool(int32_t n_inst, int64_t tiles, int32_t regions, int32_t D,
                       const dbnet_options_t& common, void* user_stream, bool any_ext,
                       bool four, int32_t emit_from) {
  if (user_stream) {
    stream = (cudaStream_t)user_stream;
    own_stream = false;
  } else {
    CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    own_stream = true;
  }
  if (n_inst < 1 || tiles < 1 || regions < 1) raise(DBNET_EINVAL, "empty engine");
  if (D < 2 || D > 256) raise(DBNET_EINVAL, "delays must be 1..255 steps");
  stride = tiles * kTile;
  if (stride >= (int64_t(1) << 31)) raise(DBNET_EINVAL, "too many neurons in one engine");
  cap_tiles = (int32_t)tiles;
  cap_R = regions;
  cap_inst = n_inst;
  inst.clear();
  inst.resize((size_t)n_inst);

  V.alloc(stride);
  J.alloc(4 * stride);
  Ibg.alloc(stride);
  fext.alloc(stride);
  ref.alloc(stride);
  // accumulators: one slot, or a ring of D slots when long delays may be
  // handed on at emission (and the ring takes at most a third of the free
  // memory)
  // (two slots at least: the pipelined schedule delivers into step g + 1's
  // slot while the update reads step g's)
  int32_t slots = 2;
  if (emit_from > 0) {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const double ring_b = (double)D * (double)stride * 8.0 * (four ? 2.0 : 1.0);
    if (ring_b <= (double)free_b / 3.0) slots = D;
    else emit_from = 0;
  }
  acc.alloc((four ? 2 : 1) * stride * (int64_t)slots);  // int2 per neuron, or int4 with four channels
  // the second stream of the pipelined schedule, ahead of the first
  {
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(cudaStreamCreateWithPriority(&stream2, cudaStreamNonBlocking, hi));
    CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
  }
  CK(cudaMemsetAsync(Ibg.p, 0, sizeof(float) * stride, stream));
  CK(cudaMemsetAsync(fext.p, 0, sizeof(float) * stride, stream));  // read only where kExtHet
  CK(cudaMemsetAsync(V.p, 0, sizeof(float) * stride, stream));
  CK(cudaMemsetAsync(J.p, 0, sizeof(float) * 4 * stride, stream));
  CK(cudaMemsetAsync(ref.p, 0, stride, stream));
  CK(cudaMemsetAsync(acc.p, 0, sizeof(int2) * (four ? 2 : 1) * stride * (size_t)slots, stream));
  if (slots > 1) {
    slot_emit.alloc(D);
    CK(cudaMemsetAsync(slot_emit.p, 0xFF, sizeof(uint16_t) * D, stream));  // none yet
  }
  desc.alloc(n_inst);
  dyn.alloc(n_inst);
  tile_info.alloc(tiles);
  closed.alloc(regions);
  region_inst.alloc(regions);
  cnt.alloc(regions);
  bw.alloc(4 * (int64_t)regions);
  ylast.alloc(regions);
  CK(cudaMemsetAsync(desc.p, 0, sizeof(InstDesc) * n_inst, stream));
  CK(cudaMemsetAsync(dyn.p, 0, sizeof(InstDyn) * n_inst, stream));  // inactive
  // host sources of the asynchronous copies that clear tiles and counters;
  // they live as long as the engine
  no_tiles_h.assign((size_t)tiles, make_int4(-1, 0, 0, 0));
  zero_dyn_h.assign((size_t)n_inst, InstDyn{});
  CK(cudaMemcpyAsync(tile_info.p, no_tiles_h.data(), sizeof(int4) * tiles, cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(region_inst.p, 0xFF, sizeof(int32_t) * regions, stream));  // -1: unused
  CK(cudaMemsetAsync(closed.p, 0, sizeof(long long) * regions, stream));
  CK(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * regions, stream));
  CK(cudaMemsetAsync(bw.p, 0, sizeof(double) * 4 * regions, stream));
  CK(cudaMemsetAsync(ylast.p, 0, sizeof(double) * regions, stream));
  // spike ring: a slot per step of the longest delay, each able to hold every neuron
  hist.alloc((int64_t)D * stride);
  hcount.alloc(D);
  CK(cudaMemsetAsync(hcount.p, 0, sizeof(uint32_t) * D, stream));
  // delay-major segment ring: room for seg_cap spikes per step -- a 64th of
  // the neurons (at least 4096), within a sixteenth of the free memory; a
  // step's spikes beyond seg_cap (and instances with u32 tables) take the
  // direct path
  const int32_t dcap = D - 1;
  int64_t seg_cap = 0;
  {
    size_t free_b = 0, total_b = 0;
    CK(cudaMemGetInfo(&free_b, &total_b));
    const int64_t budget = (int64_t)(free_b / 16);
    const int64_t per_spike = (int64_t)D * dcap * 2 + (int64_t)D * 8;
    const int64_t want = std::max<int64_t>(4096, stride / 64);
    seg_cap = std::min<int64_t>(std::min(stride, want), budget / per_spike) / 32 * 32;
    if (seg_cap < 1024) seg_cap = 0;  // too little room to be worth it
  }
  if (seg_cap > 0) {
    hseg.alloc((int64_t)D * dcap * seg_cap);
    hr0.alloc((int64_t)D * seg_cap);
  }
  base.alloc(2);
  events.alloc(2);  // [0] events counted by the deliveries, [1] scratch for the pending ones
  flags.alloc(1);
  CK(cudaMemsetAsync(base.p, 0, sizeof(unsigned long long) * 2, stream));
  CK(cudaMemsetAsync(events.p, 0, sizeof(unsigned long long), stream));
  CK(cudaMemsetAsync(flags.p, 0, sizeof(unsigned), stream));

  dev = EngineDev{};
  dev.V = V.p;
  dev.J = J.p;
  dev.Ibg = Ibg.p;
  dev.fext = fext.p;
  dev.any_ext = any_ext ? 1 : 0;
  dev.four = four ? 1 : 0;
  dev.ref = ref.p;
  dev.acc = acc.p;
  dev.stride = stride;
  dev.acc_slots = slots;
  {
    int dev_id = 0, l2 = 0;
    CK(cudaGetDevice(&dev_id));
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev_id));
    // one accumulator slot larger than a quarter of the L2: deliver in
    // rank phases, each touching about an eighth of the regions at a time
    const double slot_b = (double)stride * (four ? 16.0 : 8.0);
    dev.phases = slot_b > 0.25 * (double)l2 ? 8 : 1;
  }
  dev.d_emit = emit_from > 0 ? emit_from : D + 1;
  dev.slot_emit = slots > 1 ? slot_emit.p : nullptr;
  emit_cand = emit_from;
  emit_phase = (emit_from > 0 && common.emit_delay == 0 && common.autotune_at >= 0) ? 0 : 2;
  dev.insts = desc.p;
  dev.dyn = dyn.p;
  dev.tile_info = tile_info.p;
  dev.closed = closed.p;
  dev.cnt = cnt.p;
  dev.bw = bw.p;
  dev.ylast = ylast.p;
  dev.region_inst = region_inst.p;
  dev.hist = hist.p;
  dev.hcount = hcount.p;
  dev.hist_cap = stride;
  dev.hseg = hseg.p;
  dev.hr0 = hr0.p;
  dev.seg_cap = seg_cap;
  dev.dcap = dcap;
  dev.bin_lead = bin_lead(common);
  if (dev.bin_lead >= D - 1) raise(DBNET_EINVAL, "the spike bin is longer than the ring");
  dev.D = D;
  dev.events = events.p;
  dev.flags = flags.p;
  dev.n_inst = n_inst;
  dev.n_tiles = 0;
  dev.total_R = 0;
  n_tiles = 0;
  total_R = 0;
  del_grid = common.deliver_blocks > 0 ? common.deliver_blocks : deliver_grid();
  pbar.alloc(1);
  persist_max = persist_max_grid(dev);
  fixed_schedule = common.schedule;
  pipelined = common.schedule == DBNET_SCHEDULE_PIPELINED;
  persistent = common.schedule == DBNET_SCHEDULE_PERSISTENT;
  if (persistent) {
    if (persist_max < 2) raise(DBNET_EUNSUPPORTED, "the persistent stepper cannot be made co-resident");
    if (common.deliver_blocks > persist_max)
      raise(DBNET_EINVAL, "deliver_blocks exceeds the persistent stepper's co-resident blocks (" +
                              std::to_string(persist_max) + ")");
    del_grid = std::min(del_grid, persist_max);
  }
  if (common.autotune_at >= 0) {
    int dev_id = 0, sms = 0;
    CK(cudaGetDevice(&dev_id));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id));
    if (common.deliver_blocks > 0) {
      tune_grid.push_back(common.deliver_blocks);  // the schedule alone
    } else {
      // a few blocks only for small networks (at most two tiles per SM),
      // whose steps are all latency; 1..4 blocks per SM for every network
      if (tiles <= 2 * (int64_t)sms)
        for (int div : {8, 4, 2})
          if (sms / div >= 2) tune_grid.push_back(sms / div);
      for (int k = 1; k <= 4 && sms * k <= del_grid; ++k) tune_grid.push_back(sms * k);
    }
    // the persistent stepper only where its blocks hold at most one update
    // tile each; with more tiles it lost every measured comparison
    persist_tunable = tiles <= (int64_t)persist_max;
    tune_at = (unsigned long long)common.autotune_at;
    const size_t n_sched = fixed_schedule == DBNET_SCHEDULE_AUTO ? 3 : 1;
    if (tune_grid.size() * n_sched > 1) {
      tune_ms.assign(3 * tune_grid.size(), 0.0);  // each grid on each schedule
      tune_pending = true;
    }
  }
  CK(cudaGetLastError());
}

void Engine::place(int k, const InstSpec& sp, int32_t first_tile, int32_t rbase, int S,
                   long long n_end) {
  const GraphDev& g = *sp.graph;
  const int32_t nt = (g.N + kTile - 1) / kTile;
  if (k < 0 || k >= cap_inst || first_tile < 0 || first_tile + nt > cap_tiles || rbase < 0 ||
      rbase + g.R > cap_R)
    raise(DBNET_EINVAL, "instance placement outside the engine's capacity");
  if (g.max_delay + dev.bin_lead >= dev.D) raise(DBNET_EINVAL, "a delay is longer than the engine's ring");
  if (bin_lead(sp.opt) != dev.bin_lead) raise(DBNET_EINVAL, "spike binning differs from the engine's");
  if (g.two_w && !dev.four)
    raise(DBNET_EUNSUPPORTED, "two weights per edge need an engine with four accumulator channels");
  InstHost& ih = inst[(size_t)k];
  ih = InstHost{};
  ih.graph = sp.graph;
  ih.first_tile = first_tile;
  ih.n_tiles = nt;
  ih.rbase = rbase;
  ih.opt = sp.opt;
  ih.net_id = sp.net_id;
  for (int32_t r = 0; r < g.R; ++r)
    ih.rc_h.push_back(region_const(sp.params[r], sp.opt.dt_ms, S, g.ro_h[r], g.ro_h[r + 1],
                                   g.ro_h[r] + g.nexc_h[r]));
  ih.rc.alloc(g.R);
  CK(cudaMemcpyAsync(ih.rc.p, ih.rc_h.data(), sizeof(RegionConst) * g.R, cudaMemcpyHostToDevice, stream));
  const dbnet_options_t& o = ih.opt;
  ih.bold.alloc(std::max<int64_t>(o.bold_capacity, 1) * g.R);
  if (o.raster_capacity > 0) {
    ih.raster_step.alloc(o.raster_capacity);
    ih.raster_id.alloc(o.raster_capacity);
  }
  InstDesc d;
  std::memset(&d, 0, sizeof(d));
  d.row_ptr = g.row_ptr.p;
  d.rec = g.rec.p;
  d.two_w = g.two_w ? 1 : 0;
  d.bin_sp = sp.opt.bin_spikes ? 1 : 0;
  d.col = nullptr;
  d.w = nullptr;
  d.delay = nullptr;
  d.seg = g.seg.p;
  d.seg_kind = g.seg_kind;
  d.dmax = g.max_delay;
  d.seg_stride = g.seg_stride;
  for (const auto& p : sp.params) d.ext |= ext_bits(p);
  if (d.ext && !dev.any_ext)
    raise(DBNET_EUNSUPPORTED, "this engine was built without the OU current or injected-current factors");
  d.region_offsets = g.ro.p;
  d.rc = ih.rc.p;
  d.bold = ih.bold.p;
  d.raster_step = ih.raster_step.p;
  d.raster_id = ih.raster_id.p;
  d.base = (int64_t)first_tile * kTile;
  d.raster_cap = o.raster_capacity;
  d.bold_cap = o.bold_capacity;
  d.seed = o.seed;
  d.net_id = ih.net_id;
  d.g0 = g_host;
  d.n_end = n_end;
  d.N = g.N;
  d.R = g.R;
  d.rbase = rbase;
  d.shift = 32;
  d.tmask = 0xFFFFFFFFu;
  d.two_S = std::ldexp(1.0f, S);
  d.inv_two_S = std::ldexp(1.0f, -S);
  d.spb = (int32_t)std::lrint(o.bin_ms / o.dt_ms);
  d.bins_per_tr = (int32_t)std::lrint(o.tr_ms / o.bin_ms);
  d.h_bw = o.bin_ms * 1e-3;
  d.z_scale = o.z_scale;
  d.kappa = o.bw_kappa;
  d.gamma = o.bw_gamma;
  d.tau = o.bw_tau;
  d.alpha = o.bw_alpha;
  d.rho = o.bw_rho;
  d.V0 = o.bw_V0;
  ih.desc = d;
  // device tables: descriptor, counters, tiles and region slots
  InstDyn dy;
  std::memset(&dy, 0, sizeof(dy));
  dy.active = 1;
  std::vector<int4> ti((size_t)nt);
  for (int32_t t = 0; t < nt; ++t) {
    // regions touched by the tile's neurons [t*kTile, min((t+1)*kTile, N))
    const int32_t lo = t * kTile, hi = std::min((t + 1) * kTile, g.N) - 1;
    const int32_t r0 = (int32_t)(std::upper_bound(g.ro_h.begin(), g.ro_h.end(), lo) - g.ro_h.begin()) - 1;
    const int32_t r1 = (int32_t)(std::upper_bound(g.ro_h.begin(), g.ro_h.end(), hi) - g.ro_h.begin()) - 1;
    ti[(size_t)t] = make_int4(k, r0, r1 - r0 + 1, 0);
  }
  ih.stage_ti = std::move(ti);
  ih.stage_ri.assign((size_t)g.R, k);
  ih.stage_bw.assign((size_t)g.R * 4, 1.0);
  for (int32_t r = 0; r < g.R; ++r) ih.stage_bw[(size_t)r * 4] = 0.0;  // s = 0, f = v = q = 1
  CK(cudaMemcpyAsync(desc.p + k, &ih.desc, sizeof(InstDesc), cudaMemcpyHostToDevice, stream));
  ih.stage_dyn = dy;
  CK(cudaMemcpyAsync(dyn.p + k, &ih.stage_dyn, sizeof(InstDyn), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(tile_info.p + first_tile, ih.stage_ti.data(), sizeof(int4) * nt,
                     cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(region_inst.p + rbase, ih.stage_ri.data(), sizeof(int32_t) * g.R,
                     cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(bw.p + 4 * (int64_t)rbase, ih.stage_bw.data(), sizeof(double) * 4 * g.R,
                     cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(cnt.p + rbase, 0, sizeof(int32_t) * g.R, stream));
  CK(cudaMemsetAsync(ylast.p + rbase, 0, sizeof(double) * g.R, stream));
  CK(cudaMemsetAsync(closed.p + rbase, 0, sizeof(long long) * g.R, stream));
  launch_init_state(dev, k, nt, first_tile, stream);
  if (ih.desc.ext & kExtHet) {  // per-neuron injected-current factors
    ih.stage_fext.assign((size_t)g.N, 1.0f);
    for (int32_t r = 0; r < g.R; ++r) {
      const double kr = sp.params[(size_t)r].iext_shape;
      if (kr > 0.0)
        for (int32_t i = g.ro_h[r]; i < g.ro_h[r + 1]; ++i)
          ih.stage_fext[(size_t)i] = (float)(gamma_of(kr, sp.opt.seed, sp.net_id, i) / kr);
    }
    CK(cudaMemcpyAsync(fext.p + (int64_t)first_tile * kTile, ih.stage_fext.data(),
                       sizeof(float) * g.N, cudaMemcpyHostToDevice, stream));
  }
  CK(cudaGetLastError());
}

void Engine::vacate(int k) {
  InstHost& ih = inst[(size_t)k];
  if (!ih.graph) return;
  CK(cudaMemcpyAsync(dyn.p + k, zero_dyn_h.data() + k, sizeof(InstDyn), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(tile_info.p + ih.first_tile, no_tiles_h.data() + ih.first_tile,
                     sizeof(int4) * ih.n_tiles, cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(region_inst.p + ih.rbase, 0xFF, sizeof(int32_t) * ih.graph->R, stream));
  ih = InstHost{};  // its staged tables were copied when it was placed, long before
}

void Engine::set_extent(int32_t tiles, int32_t regions) {
  if (tiles == n_tiles && regions == total_R) return;
  if (tiles < 0 || tiles > cap_tiles || regions < 0 || regions > cap_R)
    raise(DBNET_EINVAL, "extent outside the engine's capacity");
  if (gexec) {
    CK(cudaStreamSynchronize(stream));
    CK(cudaGraphExecDestroy(gexec));
    gexec = nullptr;
  }
  n_tiles = tiles;
  total_R = regions;
  dev.n_tiles = tiles > 0 ? tiles : 1;  // one (unused) block still advances the iteration word
  dev.total_R = regions;
}

Engine::~Engine() {
  if (gexec) cudaGraphExecDestroy(gexec);
  for (auto& ev : emit_ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : tune_ev)
    if (ev) cudaEventDestroy(ev);
  if (stream2) {
    cudaStreamSynchronize(stream2);
    cudaStreamDestroy(stream2);
  }
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (own_stream && stream) {
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
  } else if (stream) {
    cudaStreamSynchronize(stream);
  }
}

void Engine::check() const {
  if (poisoned) raise(DBNET_ESTATE, "handle poisoned by an earlier failure: " + poison_msg);
}

// kChunk steps in two halves: the first half finds its iteration at
// base[0] + i and its last update writes base[1]; the second half reads
// base[1] and its last update writes base[0] for the next replay.
// kChunk steps.  Sequential: delivery then update, per step.  Pipelined:
// the short part of step g's delivery, then step g's update beside the long
// part of step g + 1's delivery (a fork onto the second stream and a join),
// so that the latency-bound delivery runs under the bandwidth-bound update;
// the replay assumes the long part of its first step is already enqueued
// and leaves the one of the step after its last enqueued.
void Engine::capture() {
  cudaGraph_t g = nullptr;
  constexpr int half = kChunk / 2;
  CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < kChunk; ++i) {
    const int h = i / half, off = i % half;
    const StepRef rd{base.p + h, (unsigned long long)off, nullptr};
    const StepRef ru{base.p + h, (unsigned long long)off, off == half - 1 ? base.p + (1 - h) : nullptr};
    if (!pipelined) {
      launch_deliver(dev, del_grid, rd, stream);
      launch_update(dev, ru, stream);
      continue;
    }
    const StepRef rn{base.p + h, (unsigned long long)off + 1ull, nullptr};  // step g + 1
    launch_deliver(dev, del_grid, rd, stream, kPartShort);
    CK(cudaEventRecord(ev_fork, stream));
    CK(cudaStreamWaitEvent(stream2, ev_fork, 0));
    launch_deliver(dev, del_grid, rn, stream2, kPartLong);
    launch_update(dev, ru, stream);
    CK(cudaEventRecord(ev_join, stream2));
    CK(cudaStreamWaitEvent(stream, ev_join, 0));
  }
  cudaError_t e1 = cudaStreamEndCapture(stream, &g);
  if (e1 != cudaSuccess) raise(DBNET_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e1));
  cudaError_t e2 = cudaGraphInstantiate(&gexec, g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) raise(DBNET_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e2));
}

void Engine::step(int64_t n) {
  check();
  if (n < 0) raise(DBNET_EINVAL, "n_steps must be >= 0");
  if (n == 0) return;
  while (n > 0) {
    const bool emit_pending = emit_phase < 2;
    if (emit_pending && g_host >= tune_at) {  // the emission threshold first,
      n -= tune_emit(n);
      continue;
    }
    if (tune_pending && g_host >= tune_at) {  // then the grid
      n -= tune_steps(n);
      continue;
    }
    const int64_t k = (tune_pending || emit_pending) ? std::min<int64_t>(n, (int64_t)(tune_at - g_host)) : n;
    run_plain(k);
    n -= k;
  }
  launch_close(dev, g_host, stream);
  CK(cudaGetLastError());
}

void Engine::set_emit(int32_t d) {
  if (d == dev.d_emit) return;
  dev.d_emit = d;
  if (gexec) {  // the captured steps carry the old threshold
    CK(cudaStreamSynchronize(stream));
    CK(cudaGraphExecDestroy(gexec));
    gexec = nullptr;
  }
}

// Up to n steps of the emission tuner: phase 0 runs without emission, phase
// 1 with the candidate threshold; each runs D steps for the spikes already
// in flight to come due under its rule, then kEmitTimed whole steps between
// two events.  The faster rule stays.  Returns the steps run.
int64_t Engine::tune_emit(int64_t n) {
  const int64_t warm = dev.D, per = warm + kEmitTimed;
  if (emit_steps == 0) set_emit(emit_phase == 0 ? dev.D + 1 : emit_cand);
  if (!emit_ev[0]) {
    CK(cudaEventCreate(&emit_ev[0]));
    CK(cudaEventCreate(&emit_ev[1]));
  }
  const int64_t k = std::min<int64_t>(n, per - emit_steps);
  int64_t ran = 0;
  while (ran < k) {
    if (emit_steps == warm) CK(cudaEventRecord(emit_ev[0], stream));
    const int64_t chunk = emit_steps < warm ? std::min<int64_t>(k - ran, warm - emit_steps) : k - ran;
    run_plain(chunk);
    ran += chunk;
    emit_steps += chunk;
  }
  if (emit_steps == per) {
    CK(cudaEventRecord(emit_ev[1], stream));
    CK(cudaEventSynchronize(emit_ev[1]));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, emit_ev[0], emit_ev[1]));
    emit_ms[emit_phase] = ms;
    emit_steps = 0;
    if (++emit_phase == 2) set_emit(emit_ms[1] < emit_ms[0] ? emit_cand : dev.D + 1);
  }
  return k;
}

// Up to n steps of the launch-shape tuner: the candidates -- a delivery grid
// and the sequential, pipelined or persistent schedule -- take turns,
// kTuneRounds times each, every turn one chunk of kChunk steps between two
// events (a captured graph, or one persistent launch, enqueued at once, so
// the timing is the device's); the
// smallest total wins, so that the network's own fluctuations of activity
// from chunk to chunk average out.  Fewer than kChunk steps run plainly and
// the tuning goes on at the next call.  Returns the steps run.
int64_t Engine::tune_steps(int64_t n) {
  const int C = (int)tune_grid.size() * 3;
  const int c = tune_done % C;
  if (n < kChunk) {
    for (int64_t i = 0; i < n; ++i) direct_step();
    return n;
  }
  const int sched = c % 3, grid = tune_grid[(size_t)(c / 3)];
  if ((fixed_schedule != DBNET_SCHEDULE_AUTO && sched + 1 != fixed_schedule) ||
      (sched == 2 && (grid > persist_max || !persist_tunable)) || tune_ms[(size_t)c] >= kDropped) {
    // not a candidate (another schedule, too many blocks to be co-resident),
    // or dropped after the first round
    tune_ms[(size_t)c] = kDropped;
    finish_turn(C);
    return 0;
  }
  set_shape(grid, sched);
  if (!pipelined && long_pending) {
    direct_step();
    return 1;
  }
  if (!gexec && !persistent) capture();
  if (pipelined && !long_pending) {
    launch_deliver(dev, del_grid, StepRef{nullptr, g_host, nullptr}, stream, kPartLong);
    long_pending = true;
  }
  if (!tune_ev[0]) {
    CK(cudaEventCreate(&tune_ev[0]));
    CK(cudaEventCreate(&tune_ev[1]));
  }
  CK(cudaEventRecord(tune_ev[0], stream));
  run_plain(kChunk);
  CK(cudaEventRecord(tune_ev[1], stream));
  CK(cudaEventSynchronize(tune_ev[1]));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, tune_ev[0], tune_ev[1]));
  tune_ms[(size_t)c] += ms;
  finish_turn(C);
  return kChunk;
}

void Engine::finish_turn(int C) {
  if (++tune_done == C) {  // after the first round, drop the candidates over twice the best
    const double best = *std::min_element(tune_ms.begin(), tune_ms.end());
    for (double& t : tune_ms)
      if (t > 2.0 * best) t = kDropped;
  }
  if (tune_done < C * kTuneRounds) return;
  int best = 0;
  for (int k = 1; k < C; ++k)
    if (tune_ms[(size_t)k] < tune_ms[(size_t)best]) best = k;
  set_shape(tune_grid[(size_t)(best / 3)], best % 3);
  tune_pending = false;
}



void Engine::set_shape(int grid, int sched) {
  if (grid == del_grid && (sched == 1) == pipelined && (sched == 2) == persistent) return;
  del_grid = grid;
  pipelined = sched == 1;
  persistent = sched == 2;
  if (gexec) {
    CK(cudaStreamSynchronize(stream));
    CK(cudaGraphExecDestroy(gexec));
    gexec = nullptr;
  }
}

// n steps with the current delivery grid: whole chunks from the captured
// graph, the rest as direct launches
void Engine::run_plain(int64_t n) {
  if (persistent) {  // the pending long part first, then whole launches
    if (n > 0 && long_pending) {
      direct_step();
      --n;
    }
    while (n > 0) {
      const int k = (int)std::min<int64_t>(n, kPersistSteps);
      CK(launch_persist(dev, del_grid, g_host, k, pbar.p, kBarrierLimitNs, stream));
      g_host += (unsigned long long)k;
      n -= k;
    }
    return;
  }
  if (n >= kChunk && !pipelined && long_pending) {  // the pending long part first
    direct_step();
    --n;
  }
  if (n >= kChunk) {
    if (!gexec) capture();
    if (pipelined && !long_pending)
      launch_deliver(dev, del_grid, StepRef{nullptr, g_host, nullptr}, stream, kPartLong);
    launch_set_base(base.p, g_host, stream);
    while (n >= kChunk) {
      CK(cudaGraphLaunch(gexec, stream));
      n -= kChunk;
      g_host += kChunk;
    }
    long_pending = pipelined;
  }
  for (; n > 0; --n) direct_step();
}

// One step by direct launches: the delivery (only its short part when the
// long part is already enqueued), then the update.
void Engine::direct_step() {
  const StepRef sr{nullptr, g_host, nullptr};
  launch_deliver(dev, del_grid, sr, stream, long_pending ? kPartShort : kPartAll);
  launch_update(dev, sr, stream);
  long_pending = false;
  ++g_host;
}

void Engine::step_timed(int64_t n, double* ms) {
  check();
  if (n < 0) raise(DBNET_EINVAL, "n_steps must be >= 0");
  constexpr int kPool = 512;  // steps per batch of events
  std::vector<cudaEvent_t> ev(3 * kPool, nullptr);
  for (auto& x : ev) CK(cudaEventCreate(&x));
  double t_del = 0.0, t_upd = 0.0;
  try {
    while (n > 0) {
      const int b = (int)std::min<int64_t>(n, kPool);
      for (int i = 0; i < b; ++i, ++g_host) {
        const StepRef sr{nullptr, g_host, nullptr};
        CK(cudaEventRecord(ev[3 * i], stream));
        launch_deliver(dev, del_grid, sr, stream, long_pending ? kPartShort : kPartAll);
        long_pending = false;
        CK(cudaEventRecord(ev[3 * i + 1], stream));
        launch_update(dev, sr, stream);
        CK(cudaEventRecord(ev[3 * i + 2], stream));
      }
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(stream));
      for (int i = 0; i < b; ++i) {
        float a = 0.f, c = 0.f;
        CK(cudaEventElapsedTime(&a, ev[3 * i], ev[3 * i + 1]));
        CK(cudaEventElapsedTime(&c, ev[3 * i + 1], ev[3 * i + 2]));
        t_del += a;
        t_upd += c;
      }
      n -= b;
    }
  } catch (...) {
    for (auto& x : ev) cudaEventDestroy(x);
    throw;
  }
  for (auto& x : ev) cudaEventDestroy(x);
  launch_close(dev, g_host, stream);
  CK(cudaGetLastError());
  ms[0] = t_del;
  ms[1] = t_upd;
}

void Engine::sync() {
  check();
  CK(cudaStreamSynchronize(stream));
  unsigned f = 0;
  CK(cudaMemcpy(&f, flags.p, sizeof(f), cudaMemcpyDeviceToHost));
  if (f & kFlagTimeout) {
    poisoned = true;
    poison_msg = "a grid barrier of the persistent stepper timed out";
    raise(DBNET_ETIMEOUT, poison_msg);
  }
  if (f & kFlagHistOverflow)
    raise(DBNET_ERANGE, "spike ring overflowed its capacity");
}

int64_t Engine::bold_samples(int k) const {
  const InstDesc& d = inst[k].desc;
  const int64_t steps = (int64_t)(g_host - d.g0);
  return steps / d.spb / d.bins_per_tr;
}

InstDyn Engine::read_dyn(int k) {
  sync();
  InstDyn d;
  CK(cudaMemcpy(&d, dyn.p + k, sizeof(d), cudaMemcpyDeviceToHost));
  return d;
}

}  // namespace dbn

// ------------------------------------------------------------------ ABI ----
using namespace dbn;


template <class F>
static int guarded(Engine* eng, F&& f) {
  try {
    f();
    return DBNET_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    if (eng && e.code == DBNET_ECUDA) {
      eng->poisoned = true;
      eng->poison_msg = e.msg;
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

extern "C" {

const char* dbnet_strerror(int code) {
  switch (code) {
    case DBNET_OK: return "ok";
    case DBNET_EINVAL: return "invalid argument";
    case DBNET_ENOMEM: return "out of memory";
    case DBNET_ECUDA: return "CUDA failure";
    case DBNET_ETIMEOUT: return "device wait timed out";
    case DBNET_EOVERFLOW: return "fixed-point accumulation could overflow";
    case DBNET_ESTATE: return "handle poisoned by an earlier failure";
    case DBNET_ERANGE: return "capacity exceeded";
    case DBNET_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

const char* dbnet_last_error(void) { return g_last_error.c_str(); }

int dbnet_abi_sizes(int64_t* out, int n) {
  const int64_t sz[11] = {
      (int64_t)sizeof(dbnet_graph_t),   (int64_t)sizeof(dbnet_region_params_t),
      (int64_t)sizeof(dbnet_options_t), (int64_t)sizeof(dbnet_stats_t),
      (int64_t)sizeof(dbens_enkf_t),    (int64_t)sizeof(dbnet_device_graph_t),
      (int64_t)sizeof(dbsrv_options_t), (int64_t)sizeof(dbsrv_request_t),
      (int64_t)sizeof(dbsrv_status_t),  (int64_t)sizeof(dbsrv_stats_t),
      0};
  if (!out && n > 0) return DBNET_EINVAL;
  for (int k = 0; k < n && k < 11; ++k) out[k] = sz[k];
  return 10;
}

int dbnet_barrier_probe(int32_t blocks, int32_t missing, int32_t rounds, int64_t limit_us) {
  return guarded(nullptr, [&] {
    int dev_id = 0, sms = 0;
    CK(cudaGetDevice(&dev_id));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id));
    if (blocks < 1 || blocks > sms || missing < 0 || rounds < 1 || limit_us < 1 || limit_us > 10000000)
      raise(DBNET_EINVAL, "barrier probe: blocks in 1..SMs, missing >= 0, rounds >= 1, limit_us in 1..1e7");
    DevBuf<unsigned> w;  // the barrier's count and the flags word
    w.alloc(2);
    CK(cudaMemset(w.p, 0, 2 * sizeof(unsigned)));
    CK(launch_barrier_probe(blocks, (unsigned)missing, rounds, (unsigned long long)limit_us * 1000ull,
                            w.p, w.p + 1, nullptr));
    CK(cudaStreamSynchronize(nullptr));
    unsigned f = 0;
    CK(cudaMemcpy(&f, w.p + 1, sizeof(f), cudaMemcpyDeviceToHost));
    if (f & kFlagTimeout) raise(DBNET_ETIMEOUT, "the grid barrier's wait gave up at its limit");
  });
}

int dbnet_set_allocator(const dbnet_allocator_t* a) {
  std::lock_guard<std::mutex> lock(g_hook_mu);
  if (a && ((a->alloc == nullptr) != (a->free == nullptr))) {
    g_last_error = "an allocator needs both alloc and free";
    return DBNET_EINVAL;
  }
  g_hook = (a && a->alloc) ? AllocHook{a->alloc, a->free, a->ctx} : AllocHook{};
  return DBNET_OK;
}

int dbnet_options_default(dbnet_options_t* o) {
  if (!o) return DBNET_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->dt_ms = 0.1;
  o->bin_ms = 1.0;
  o->tr_ms = 800.0;
  o->z_scale = 1.0;
  o->bw_kappa = 0.65;
  o->bw_gamma = 0.41;
  o->bw_tau = 0.98;
  o->bw_alpha = 0.32;
  o->bw_rho = 0.34;
  o->bw_V0 = 0.02;
  o->seed = 1;
  o->net_id = 0;
  o->fixed_shift = 0;
  o->precision = 32;
  o->raster_capacity = 0;
  o->bold_capacity = 4096;
  o->autotune_at = 2000;
  o->emit_delay = -1;
  return DBNET_OK;
}

int dbnet_create(const dbnet_graph_t* graph, const dbnet_region_params_t* params,
                 const dbnet_options_t* options, void* cuda_stream, dbnet_t** out) {
  if (out) *out = nullptr;
  std::unique_ptr<dbnet> h(new (std::nothrow) dbnet());
  if (!h) return DBNET_ENOMEM;
  int rc = guarded(nullptr, [&] {
    AllocStreamScope alloc_stream(cuda_stream);
    if (!out || !params || !options) raise(DBNET_EINVAL, "NULL argument");
    check_options(*options);
    if (!graph) raise(DBNET_EINVAL, "graph is NULL");
    if (graph->n_regions < 1) raise(DBNET_EINVAL, "n_regions must be >= 1");
    for (int32_t r = 0; r < graph->n_regions; ++r)
      check_params(params[r], options->dt_ms, bin_lead(*options));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    auto g = upload_graph(graph, s);
    InstSpec sp;
    sp.graph = g;
    sp.params.assign(params, params + graph->n_regions);
    sp.opt = *options;
    sp.net_id = options->net_id;
    h->own.reset(new Engine());
    h->eng = h->own.get();
    h->eng->init({sp}, cuda_stream);
  });
  if (rc == DBNET_OK) *out = h.release();
  return rc;
}

int dbnet_step(dbnet_t* h, int64_t n_steps) {
  if (!h || !h->own) return DBNET_EINVAL;
  return guarded(h->eng, [&] { h->eng->step(n_steps); });
}

int dbnet_step_timed(dbnet_t* h, int64_t n_steps, double* ms) {
  if (!h || !h->own || !ms) return DBNET_EINVAL;
  return guarded(h->eng, [&] { h->eng->step_timed(n_steps, ms); });
}

int dbnet_sync(dbnet_t* h) {
  if (!h) return DBNET_EINVAL;
  return guarded(h->eng, [&] { h->eng->sync(); });
}

int dbnet_read_spikes(dbnet_t* h, int64_t t0, int64_t t1, int32_t* step, int32_t* id, int64_t cap,
                      int64_t* n_out) {
  if (!h || !n_out || cap < 0 || (cap > 0 && (!step || !id))) return DBNET_EINVAL;
  *n_out = 0;
  int64_t matched = 0;
  int rc = guarded(h->eng, [&] {
    Engine& e = *h->eng;
    const InstHost& ih = e.inst[h->inst];
    InstDyn d = e.read_dyn(h->inst);
    const int64_t n = std::min<int64_t>((int64_t)d.raster_count, ih.opt.raster_capacity);
    std::vector<int32_t> s((size_t)n), i((size_t)n);
    if (n > 0) {
      CK(cudaMemcpy(s.data(), ih.raster_step.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(i.data(), ih.raster_id.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    }
    std::vector<uint64_t> key;
    key.reserve((size_t)n);
    for (int64_t k = 0; k < n; ++k)
      if (s[(size_t)k] >= t0 && s[(size_t)k] < t1)
        key.push_back(((uint64_t)(uint32_t)s[(size_t)k] << 32) | (uint32_t)i[(size_t)k]);
    std::sort(key.begin(), key.end());
    matched = (int64_t)key.size();
    const int64_t w = std::min<int64_t>(matched, cap);
    for (int64_t k = 0; k < w; ++k) {
      step[k] = (int32_t)(key[(size_t)k] >> 32);
      id[k] = (int32_t)(key[(size_t)k] & 0xFFFFFFFFu);
    }
    *n_out = w;
  });
  if (rc == DBNET_OK && matched > cap) {
    g_last_error = "more spikes match than cap";
    return DBNET_ERANGE;
  }
  return rc;
}

int dbnet_read_bold(dbnet_t* h, double* y, int64_t cap_samples, int64_t* n_out) {
  if (!h || !n_out || cap_samples < 0 || (cap_samples > 0 && !y)) return DBNET_EINVAL;
  *n_out = 0;
  return guarded(h->eng, [&] {
    Engine& e = *h->eng;
    const InstHost& ih = e.inst[h->inst];
    InstDyn d = e.read_dyn(h->inst);
    (void)d;
    const int64_t avail = std::min<int64_t>(e.bold_samples(h->inst), ih.opt.bold_capacity);
    const int64_t n = std::min(avail, cap_samples);
    if (n > 0)
      CK(cudaMemcpy(y, ih.bold.p, sizeof(double) * n * ih.graph->R, cudaMemcpyDeviceToHost));
    *n_out = n;
  });
}

int dbnet_read_bw(dbnet_t* h, double* x) {
  if (!h || !x) return DBNET_EINVAL;
  return guarded(h->eng, [&] {
    Engine& e = *h->eng;
    e.sync();
    const InstHost& ih = e.inst[h->inst];
    CK(cudaMemcpy(x, e.bw.p + 4 * ih.rbase, sizeof(double) * 4 * ih.graph->R, cudaMemcpyDeviceToHost));
  });
}

int dbnet_read_state(dbnet_t* h, float* V, float* J, int32_t* ref) {
  if (!h) return DBNET_EINVAL;
  return guarded(h->eng, [&] {
    Engine& e = *h->eng;
    e.sync();
    const InstHost& ih = e.inst[h->inst];
    const int64_t base = (int64_t)ih.first_tile * kTile;
    const int32_t N = ih.graph->N;
    if (V) CK(cudaMemcpy(V, e.V.p + base, sizeof(float) * N, cudaMemcpyDeviceToHost));
    if (J)
      for (int u = 0; u < 4; ++u)
        CK(cudaMemcpy(J + (int64_t)u * N, e.J.p + u * e.stride + base, sizeof(float) * N,
                      cudaMemcpyDeviceToHost));
    if (ref) {
      std::vector<uint8_t> r((size_t)N);
      CK(cudaMemcpy(r.data(), e.ref.p + base, N, cudaMemcpyDeviceToHost));
      for (int32_t i = 0; i < N; ++i) ref[i] = r[(size_t)i];
    }
  });
}

int dbnet_set_state(dbnet_t* h, const float* V, const float* J, const int32_t* ref) {
  if (!h || !h->own) return DBNET_EINVAL;
  return guarded(h->eng, [&] {
    Engine& e = *h->eng;
    e.sync();
    const InstHost& ih = e.inst[h->inst];
    const int64_t base = (int64_t)ih.first_tile * kTile;
    const int32_t N = ih.graph->N;
    std::vector<uint8_t> r;
    if (ref) {
      r.resize((size_t)N);
      for (int32_t i = 0; i < N; ++i) {
        if (ref[i] < 0 || ref[i] > 255) raise(DBNET_EINVAL, "ref values must be in 0..255");
        r[(size_t)i] = (uint8_t)ref[i];
      }
    }
    if (V) CK(cudaMemcpy(e.V.p + base, V, sizeof(float) * N, cudaMemcpyHostToDevice));
    if (J)
      for (int u = 0; u < 4; ++u)
        CK(cudaMemcpy(e.J.p + u * e.stride + base, J + (int64_t)u * N, sizeof(float) * N,
                      cudaMemcpyHostToDevice));
    if (ref) CK(cudaMemcpy(e.ref.p + base, r.data(), N, cudaMemcpyHostToDevice));
  });
}

int dbnet_read_ibg(dbnet_t* h, float* I_bg) {
  if (!h || !I_bg) return DBNET_EINVAL;
  return guarded(h->eng, [&] {
    Engine& e = *h->eng;
    e.sync();
    const InstHost& ih = e.inst[h->inst];
    CK(cudaMemcpy(I_bg, e.Ibg.p + (int64_t)ih.first_tile * kTile, sizeof(float) * ih.graph->N,
                  cudaMemcpyDeviceToHost));
  });
}

int dbnet_set_ibg(dbnet_t* h, const float* I_bg) {
  if (!h || !h->own || !I_bg) return DBNET_EINVAL;
  return guarded(h->eng, [&] {
    Engine& e = *h->eng;
    e.sync();
    const InstHost& ih = e.inst[h->inst];
    CK(cudaMemcpy(e.Ibg.p + (int64_t)ih.first_tile * kTile, I_bg, sizeof(float) * ih.graph->N,
                  cudaMemcpyHostToDevice));
  });
}

int dbnet_stats(dbnet_t* h, dbnet_stats_t* out) {
  if (!h || !out) return DBNET_EINVAL;
  return guarded(h->eng, [&] {
    Engine& e = *h->eng;
    const InstHost& ih = e.inst[h->inst];
    InstDyn d = e.read_dyn(h->inst);
    // the deliveries count a spike's events at its delay-1 item; those of
    // the spikes handed on at the last step are added here
    CK(cudaMemsetAsync(e.events.p + 1, 0, sizeof(unsigned long long), e.stream));
    launch_pending_events(e.dev, e.g_host, e.events.p + 1, e.stream);
    CK(cudaGetLastError());
    unsigned long long evs[2] = {0, 0};
    CK(cudaMemcpyAsync(evs, e.events.p, sizeof(evs), cudaMemcpyDeviceToHost, e.stream));
    CK(cudaStreamSynchronize(e.stream));
    const unsigned long long ev = evs[0] + evs[1];
    std::memset(out, 0, sizeof(*out));
    out->step = (int64_t)(e.g_host - ih.desc.g0);
    out->spikes = (int64_t)d.spikes;
    out->events = (int64_t)ev;
    const int64_t cap = ih.opt.raster_capacity;
    out->raster_len = std::min<int64_t>((int64_t)d.raster_count, cap);
    out->raster_dropped = std::max<int64_t>((int64_t)d.raster_count - cap, 0);
    out->bold_samples = std::min<int64_t>(e.bold_samples(h->inst), ih.opt.bold_capacity);
    out->fixed_shift = e.shift_S;
    out->max_delay = ih.graph->max_delay;
    out->packed_edges = ih.graph->packed ? 1 : 0;
    out->weights_rounded = ih.graph->rounded ? 1 : 0;
    out->deliver_blocks = e.del_grid;
    out->seg_ring = ih.graph->seg_kind == kSeg16 ? (int32_t)e.dev.seg_cap : 0;
    out->emit_delay = e.dev.d_emit <= e.dev.D ? e.dev.d_emit : 0;
    out->schedule = e.persistent ? DBNET_SCHEDULE_PERSISTENT
                   : e.pipelined ? DBNET_SCHEDULE_PIPELINED : DBNET_SCHEDULE_SEQUENTIAL;
    out->autotuned = (!e.tune_pending && !e.tune_grid.empty()) ? 1 : 0;
    out->two_weights = e.dev.four;
  });
}

void dbnet_destroy(dbnet_t* h) {
  if (!h || !h->own) return;  // member views belong to their ensemble
  delete h;
}

}  // extern "C"

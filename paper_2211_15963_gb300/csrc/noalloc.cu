// dbnet_run_noalloc: a run of one network that allocates nothing.
//
// Who needs it: callers that may not allocate device memory while they run
// (a framework arena that owns every byte of the GPU, a real-time loop that
// cannot afford cudaMalloc's implicit synchronisation).  They pass the graph
// and the output state in device memory they already own; everything else
// the kernels need lives in one static device array defined below, whose
// size is fixed at DBNET_NOALLOC_SCRATCH_BYTES and which every GPU that loads
// the library keeps until the process exits.
//
// The name g_noalloc_scratch is only a host-side stand-in: host code must
// never hand it to a kernel.  The device address is looked up once per device
// with cudaGetSymbolAddress (with that device current) and cached.
//
// The same kernels as dbnet_step run here (init, deliver, update), so results
// are identical to dbnet_create + dbnet_step on the same graph and options.
// All calls share the scratch; each call clears it first; overlapping calls
// race.  Without room for a per-graph segment table, the delivery finds each
// spike's due segment by binary search over its row's delays.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "dbnet.h"
#include "engine.h"
#include "host.h"

namespace dbn {

int choose_shift(const GraphDev& g, double wext_max, int32_t requested);

namespace {

constexpr int kMaxN = DBNET_NOALLOC_MAX_NEURONS;
constexpr int kMaxR = DBNET_NOALLOC_MAX_REGIONS;
constexpr uint64_t kMaxLive = DBNET_NOALLOC_MAX_LIVE;
constexpr int kMaxTiles = kMaxN / kTile;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets inside the scratch array.
constexpr size_t kOffHist = 0;  // spike ring: kMaxLive entries
constexpr size_t kOffAcc = align256(kOffHist + sizeof(uint32_t) * kMaxLive);
constexpr size_t kOffIndeg = align256(kOffAcc + sizeof(int2) * kMaxN);
constexpr size_t kOffRc = align256(kOffIndeg + sizeof(int32_t) * kMaxN);
constexpr size_t kOffRo = align256(kOffRc + sizeof(RegionConst) * kMaxR);
constexpr size_t kOffDesc = align256(kOffRo + sizeof(int32_t) * (kMaxR + 1));
constexpr size_t kOffDyn = align256(kOffDesc + sizeof(InstDesc));
constexpr size_t kOffTiles = align256(kOffDyn + sizeof(InstDyn));
constexpr size_t kOffRegInst = align256(kOffTiles + sizeof(int4) * kMaxTiles);
constexpr size_t kOffCnt = align256(kOffRegInst + sizeof(int32_t) * kMaxR);
constexpr size_t kOffBw = align256(kOffCnt + sizeof(int32_t) * kMaxR);
constexpr size_t kOffYlast = align256(kOffBw + sizeof(double) * 4 * kMaxR);
constexpr size_t kOffHcount = align256(kOffYlast + sizeof(double) * kMaxR);  // uint32[256]
constexpr size_t kOffClosed = align256(kOffHcount + sizeof(uint32_t) * 256);  // int64[kMaxR]
constexpr size_t kOffEvents = align256(kOffClosed + sizeof(long long) * kMaxR);
constexpr size_t kOffFlags = align256(kOffEvents + sizeof(unsigned long long));
constexpr size_t kOffScal = align256(kOffFlags + sizeof(unsigned));          // uint32[4]
constexpr size_t kScratchUsed = align256(kOffScal + sizeof(unsigned) * 4);
// everything from kOffAcc on is cleared at the start of every call
constexpr size_t kClearFrom = kOffAcc;

static_assert(kScratchUsed <= DBNET_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds its size");

}  // namespace
}  // namespace dbn

// The scratch itself: file scope, fixed size, 256-byte aligned.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DBNET_NOALLOC_SCRATCH_BYTES];

namespace dbn {
namespace {

std::mutex g_scratch_mu;
unsigned char* g_scratch_addr[256] = {nullptr};

// Device address of the scratch on the current device (looked up once).
unsigned char* scratch_on_current_device() {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) raise(DBNET_EUNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      raise(DBNET_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  return g_scratch_addr[dev];
}

// Read-only check of a caller's device graph: row_ptr starts at 0 and does
// not decrease, targets lie in [0, N), delays are 1..255 and non-decreasing
// within each row, BF16 weights are finite and non-negative.  Also counts
// in-degrees and the largest weight and delay.  Warp per row.
__global__ void k_validate_ro(int32_t N, const int64_t* __restrict__ row_ptr,
                              const int32_t* __restrict__ col, const uint16_t* __restrict__ w,
                              const uint8_t* __restrict__ delay, int32_t* indeg,
                              unsigned* scal /* wmax bits, dmax, err, - */) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned err = 0, wmax = 0, dmax = 0;
  for (int64_t j = warp; j < N; j += nwarps) {
    const int64_t a = row_ptr[j], b = row_ptr[j + 1];
    if (j == 0 && a != 0) err |= kErrTarget;
    if (b < a) {
      err |= kErrTarget;
      continue;
    }
    for (int64_t e0 = a; e0 < b; e0 += 32) {
      const int64_t e = e0 + lane;
      if (e >= b) continue;
      const int32_t t = col[e];
      const unsigned d = delay[e];
      if (t < 0 || t >= N) err |= kErrTarget;
      else atomicAdd(indeg + t, 1);
      if (d < 1u) err |= kErrDelayRange;
      if (e > a && delay[e - 1] > d) err |= kErrDelayOrder;
      const uint32_t wu = (uint32_t)w[e] << 16;
      const float wf = __uint_as_float(wu);
      if (!(wf >= 0.0f) || isinf(wf)) err |= kErrWeight;
      else wmax = max(wmax, wu);
      dmax = max(dmax, d);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    err |= __shfl_xor_sync(0xffffffffu, err, o);
    wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  }
  if (lane == 0) {
    if (err) atomicOr(scal + 2, err);
    atomicMax(scal + 0, wmax);
    atomicMax(scal + 1, dmax);
  }
}

}  // namespace
}  // namespace dbn

using namespace dbn;

extern "C" int dbnet_run_noalloc(const dbnet_device_graph_t* graph,
                                 const dbnet_region_params_t* params,
                                 const dbnet_options_t* options, int64_t n_steps, float* V,
                                 float* J, uint8_t* ref, int32_t* raster_step, int32_t* raster_id,
                                 int64_t raster_cap, int64_t* n_spikes, int64_t* n_events,
                                 void* cuda_stream) {
  try {
    if (!graph || !params || !options || !V || !J || !ref || !n_spikes || !n_events)
      raise(DBNET_EINVAL, "NULL argument");
    if (n_steps < 0 || raster_cap < 0 || (raster_cap > 0 && (!raster_step || !raster_id)))
      raise(DBNET_EINVAL, "bad step count or raster buffers");
    // the update kernel moves whole tiles of V, J and ref with 16-byte bulk copies
    if ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(J) |
         reinterpret_cast<uintptr_t>(ref)) & 15u)
      raise(DBNET_EINVAL, "V, J and ref must be 16-byte aligned");
    const int32_t N = graph->n_neurons, R = graph->n_regions;
    if (N < 1 || R < 1 || !graph->region_offsets || !graph->n_exc || !graph->row_ptr ||
        !graph->col || !graph->weight_bf16 || !graph->delay)
      raise(DBNET_EINVAL, "incomplete graph");
    if (N > kMaxN)
      raise(DBNET_ERANGE, "n_neurons " + std::to_string(N) + " exceeds the allocation-free limit " +
                              std::to_string(kMaxN));
    if (R > kMaxR)
      raise(DBNET_ERANGE, "n_regions " + std::to_string(R) + " exceeds the allocation-free limit " +
                              std::to_string(kMaxR));
    const int32_t* ro = graph->region_offsets;
    if (ro[0] != 0 || ro[R] != N) raise(DBNET_EINVAL, "region_offsets must run from 0 to n_neurons");
    for (int32_t r = 0; r < R; ++r) {
      if (ro[r + 1] - ro[r] < 1) raise(DBNET_EINVAL, "region_offsets must be strictly increasing");
      if (graph->n_exc[r] < 0 || graph->n_exc[r] > ro[r + 1] - ro[r]) raise(DBNET_EINVAL, "n_exc out of range");
    }
    check_options(*options);
    if (options->bin_spikes)
      raise(DBNET_EUNSUPPORTED, "the allocation-free entry point hands every spike on in its own step");
    for (int32_t r = 0; r < R; ++r) {
      check_params(params[r], options->dt_ms, 0);
      if (params[r].ou_mu != 0.0 || params[r].ou_sigma != 0.0 || params[r].iext_shape != 0.0)
        raise(DBNET_EUNSUPPORTED,
              "the allocation-free entry point has no OU state or injected-current factors");
    }

    cudaStream_t s = (cudaStream_t)cuda_stream;
    unsigned char* base = scratch_on_current_device();
    auto at = [&](size_t off) { return base + off; };
    const int n_tiles = (N + kTile - 1) / kTile;
    const int64_t n_pad = (int64_t)n_tiles * kTile;

    // clear everything a run must start from zero, then validate the graph
    CK(cudaMemsetAsync(at(kClearFrom), 0, kScratchUsed - kClearFrom, s));
    int32_t* indeg = reinterpret_cast<int32_t*>(at(kOffIndeg));
    unsigned* scal = reinterpret_cast<unsigned*>(at(kOffScal));
    k_validate_ro<<<std::max(1, std::min(152 * 16, (N * 32 + 255) / 256)), 256, 0, s>>>(
        N, graph->row_ptr, graph->col, graph->weight_bf16, graph->delay, indeg, scal);
    launch_max_reduce(indeg, N, scal + 3, s);
    CK(cudaGetLastError());
    unsigned h[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(h, scal, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[2] & kErrTarget) raise(DBNET_EINVAL, "row_ptr or an edge target is invalid");
    if (h[2] & kErrDelayRange) raise(DBNET_EINVAL, "an edge delay is 0");
    if (h[2] & kErrDelayOrder) raise(DBNET_EINVAL, "delays must be non-decreasing within each row");
    if (h[2] & kErrWeight) raise(DBNET_EINVAL, "weights must be finite and non-negative");
    const int32_t dmax = (int32_t)std::max(1u, h[1]);

    // fixed-point scale by the same rule as dbnet_create
    GraphDev gd;
    gd.N = N;
    gd.R = R;
    gd.kin_max = (int32_t)h[3];
    float wmax;
    std::memcpy(&wmax, &h[0], 4);
    gd.w_max = (double)wmax;
    double wext_max = 0.0;
    for (int32_t r = 0; r < R; ++r) wext_max = std::max(wext_max, params[r].w_ext);
    const int S = choose_shift(gd, wext_max, options->fixed_shift);

    // region constants and the spike-ring bound (a slot per step of the
    // longest delay, each able to hold every neuron)
    RegionConst rc[kMaxR];
    for (int32_t r = 0; r < R; ++r)
      rc[r] = region_const(params[r], options->dt_ms, S, ro[r], ro[r + 1], ro[r] + graph->n_exc[r]);
    const uint64_t ring = (uint64_t)n_pad * (uint64_t)(dmax + 1);
    if (ring > kMaxLive)
      raise(DBNET_ERANGE, "a spike ring of " + std::to_string(ring) +
                              " entries (padded neurons x (longest delay + 1)) is above the "
                              "allocation-free limit " + std::to_string(kMaxLive));

    InstDesc d;
    std::memset(&d, 0, sizeof(d));
    d.row_ptr = graph->row_ptr;
    d.col = reinterpret_cast<const uint32_t*>(graph->col);
    d.w = graph->weight_bf16;
    d.delay = graph->delay;  // separate delay array: targets are used as given
    d.seg = nullptr;         // segments found by binary search over each row's delays
    d.seg_kind = kSegSearch;
    d.dmax = dmax;
    d.region_offsets = reinterpret_cast<const int32_t*>(at(kOffRo));
    d.rc = reinterpret_cast<const RegionConst*>(at(kOffRc));
    d.bold = nullptr;
    d.bold_cap = 0;
    d.raster_step = raster_step;
    d.raster_id = raster_id;
    d.raster_cap = raster_cap;
    d.base = 0;
    d.seed = options->seed;
    d.net_id = options->net_id;
    d.n_end = LLONG_MAX;  // runs every step it is given
    d.N = N;
    d.R = R;
    d.rbase = 0;
    d.shift = 32;
    d.tmask = 0xFFFFFFFFu;
    d.two_S = std::ldexp(1.0f, S);
    d.inv_two_S = std::ldexp(1.0f, -S);
    d.spb = (int32_t)std::lrint(options->bin_ms / options->dt_ms);
    d.bins_per_tr = (int32_t)std::lrint(options->tr_ms / options->bin_ms);
    d.h_bw = options->bin_ms * 1e-3;
    d.z_scale = options->z_scale;
    d.kappa = options->bw_kappa;
    d.gamma = options->bw_gamma;
    d.tau = options->bw_tau;
    d.alpha = options->bw_alpha;
    d.rho = options->bw_rho;
    d.V0 = options->bw_V0;
    InstDyn dyn;
    std::memset(&dyn, 0, sizeof(dyn));
    dyn.active = 1;
    double bw[4 * kMaxR];
    for (int32_t r = 0; r < R; ++r) {
      bw[4 * r] = 0.0;
      bw[4 * r + 1] = bw[4 * r + 2] = bw[4 * r + 3] = 1.0;
    }
    // per tile: instance 0, first region, regions touched; region owners stay 0
    int4 tiles[kMaxTiles];
    for (int t = 0; t < n_tiles; ++t) {
      const int32_t lo = t * kTile, hi = std::min((t + 1) * kTile, N) - 1;
      int32_t r0 = 0, r1 = 0;
      while (ro[r0 + 1] <= lo) ++r0;
      r1 = r0;
      while (ro[r1 + 1] <= hi) ++r1;
      tiles[t] = make_int4(0, r0, r1 - r0 + 1, 0);
    }
    CK(cudaMemcpyAsync(at(kOffTiles), tiles, sizeof(int4) * n_tiles, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(at(kOffRc), rc, sizeof(RegionConst) * R, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(at(kOffRo), ro, sizeof(int32_t) * (R + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(at(kOffDesc), &d, sizeof(d), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(at(kOffDyn), &dyn, sizeof(dyn), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(at(kOffBw), bw, sizeof(double) * 4 * R, cudaMemcpyHostToDevice, s));

    EngineDev e{};
    e.V = V;
    e.J = J;
    e.ref = ref;
    e.acc = reinterpret_cast<int2*>(at(kOffAcc));
    e.stride = n_pad;
    e.acc_slots = 1;
    e.phases = 1;
    e.d_emit = dmax + 2;  // every delay at arrival time
    e.slot_emit = nullptr;
    e.insts = reinterpret_cast<const InstDesc*>(at(kOffDesc));
    e.dyn = reinterpret_cast<InstDyn*>(at(kOffDyn));
    e.tile_info = reinterpret_cast<const int4*>(at(kOffTiles));
    e.closed = reinterpret_cast<long long*>(at(kOffClosed));
    e.cnt = reinterpret_cast<int32_t*>(at(kOffCnt));
    e.bw = reinterpret_cast<double*>(at(kOffBw));
    e.ylast = reinterpret_cast<double*>(at(kOffYlast));
    e.region_inst = reinterpret_cast<const int32_t*>(at(kOffRegInst));
    e.hist = reinterpret_cast<uint32_t*>(at(kOffHist));
    e.hcount = reinterpret_cast<uint32_t*>(at(kOffHcount));
    e.hist_cap = n_pad;
    e.D = dmax + 1;
    e.events = reinterpret_cast<unsigned long long*>(at(kOffEvents));
    e.flags = reinterpret_cast<unsigned*>(at(kOffFlags));
    e.n_inst = 1;
    e.n_tiles = n_tiles;
    e.total_R = R;

    launch_init_state(e, 0, n_tiles, 0, s);
    const int grid = deliver_grid();
    for (int64_t k = 0; k < n_steps; ++k) {
      const StepRef sr{nullptr, (unsigned long long)k, nullptr};
      launch_deliver(e, grid, sr, s);
      launch_update(e, sr, s);
    }
    launch_close(e, (unsigned long long)n_steps, s);
    // the last step's spikes: their events, not yet reached by a delivery
    launch_pending_events(e, (unsigned long long)n_steps, e.events, s);
    CK(cudaGetLastError());
    InstDyn out_dyn;
    unsigned long long ev = 0;
    unsigned flags = 0;
    CK(cudaMemcpyAsync(&out_dyn, at(kOffDyn), sizeof(out_dyn), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&ev, at(kOffEvents), sizeof(ev), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&flags, at(kOffFlags), sizeof(flags), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (flags & kFlagHistOverflow) raise(DBNET_ERANGE, "spike ring overflowed");
    *n_spikes = (int64_t)out_dyn.spikes;
    *n_events = (int64_t)ev;
    return DBNET_OK;
  } catch (const Error& err) {
    g_last_error = err.msg;
    return err.code;
  } catch (...) {
    g_last_error = "unexpected failure";
    return DBNET_ECUDA;
  }
}

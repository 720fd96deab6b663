// Host-side engine types shared by engine.cu and ens.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <iterator>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "dbnet.h"
#include "engine.h"
#include "freelist.h"

namespace dbn {

struct Error {
  int code;
  std::string msg;
};

[[noreturn]] inline void raise(int code, const std::string& msg) { throw Error{code, msg}; }

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t _e = (call);                                                          \
    if (_e != cudaSuccess)                                                            \
      ::dbn::raise(_e == cudaErrorMemoryAllocation ? DBNET_ENOMEM : DBNET_ECUDA,      \
                   std::string(#call) + ": " + cudaGetErrorString(_e));               \
  } while (0)

extern thread_local std::string g_last_error;

// The caller's device allocator (dbnet_set_allocator), or none (cudaMalloc).
// Each allocation keeps the hook it came from, so that it is returned to the
// same allocator whatever is installed later.
struct AllocHook {
  dbnet_alloc_fn alloc = nullptr;
  dbnet_free_fn free = nullptr;
  void* ctx = nullptr;
};
AllocHook current_alloc_hook();
// The stream handed to the hook: the handle's stream while a handle is
// being built or destroyed on this thread.
extern thread_local void* g_alloc_stream;
struct AllocStreamScope {
  void* prev;
  explicit AllocStreamScope(void* s) : prev(g_alloc_stream) { g_alloc_stream = s; }
  ~AllocStreamScope() { g_alloc_stream = prev; }
};

// Device memory from the hook when one is installed, else cudaMalloc.
inline void* dev_alloc(size_t bytes, AllocHook& used, void*& stream_used, const char* what) {
  const AllocHook h = current_alloc_hook();
  if (h.alloc) {
    void* p = h.alloc(bytes, g_alloc_stream, h.ctx);
    if (!p) raise(DBNET_ENOMEM, std::string("the installed allocator returned NULL for ") +
                                    std::to_string(bytes) + " bytes of " + what);
    used = h;
    stream_used = g_alloc_stream;
    return p;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    raise(e == cudaErrorMemoryAllocation ? DBNET_ENOMEM : DBNET_ECUDA,
          "cudaMalloc of " + std::to_string(bytes) + " bytes of " + what + ": " +
              cudaGetErrorString(e));
  }
  used = AllocHook{};
  stream_used = nullptr;
  return p;
}
inline void dev_free(void* p, size_t bytes, const AllocHook& used, void* stream_used) {
  if (!p) return;
  if (used.free) used.free(p, bytes, stream_used, used.ctx);
  else cudaFree(p);
}

// A sub-allocator over one device allocation (first fit, 256-byte granules,
// neighbours merged on release).  Used by the request server, so that
// admitting and retiring requests never calls cudaMalloc or cudaFree (the
// latter waits for the whole device).  Not thread-safe.
class Arena {
 public:
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  ~Arena() { dev_free(base_, (size_t)size_, hook_, hook_stream_); }
  void init(int64_t bytes) {
    bytes = round(bytes);
    base_ = static_cast<char*>(dev_alloc((size_t)bytes, hook_, hook_stream_, "the request arena"));
    size_ = bytes;
    free_.reset(bytes);
  }
  void* take(int64_t bytes) {
    bytes = round(bytes);
    const int64_t off = free_.take(bytes);
    if (off < 0) return nullptr;
    used_ += bytes;
    return base_ + off;
  }
  void give(void* p, int64_t bytes) {
    bytes = round(bytes);
    used_ -= bytes;
    free_.give(static_cast<char*>(p) - base_, bytes);
  }
  int64_t largest_free() const { return free_.largest(); }
  int64_t used() const { return used_; }
  int64_t size() const { return size_; }
  static int64_t round(int64_t b) { return (b + 255) / 256 * 256; }

 private:
  char* base_ = nullptr;
  int64_t size_ = 0, used_ = 0;
  FreeList<int64_t> free_;  // byte offsets
  AllocHook hook_;
  void* hook_stream_ = nullptr;
};

// The arena DevBuf::alloc draws from on this thread (nullptr: cudaMalloc).
extern thread_local Arena* g_arena;
struct ArenaScope {
  Arena* prev;
  explicit ArenaScope(Arena* a) : prev(g_arena) { g_arena = a; }
  ~ArenaScope() { g_arena = prev; }
};

// Device allocation owned by its holder: cudaMalloc memory, or a range of
// the arena that was current when it was allocated.
template <class T>
struct DevBuf {
  T* p = nullptr;
  int64_t n = 0;
  Arena* ar = nullptr;
  AllocHook hk;        // the allocator the memory came from (none: cudaMalloc)
  void* hk_stream = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), ar(o.ar), hk(o.hk), hk_stream(o.hk_stream) {
    o.p = nullptr; o.n = 0; o.ar = nullptr;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      reset();
      p = o.p; n = o.n; ar = o.ar; hk = o.hk; hk_stream = o.hk_stream;
      o.p = nullptr; o.n = 0; o.ar = nullptr;
    }
    return *this;
  }
  ~DevBuf() { reset(); }
  void alloc(int64_t count) {
    reset();
    if (count <= 0) return;
    const size_t bytes = sizeof(T) * (size_t)count;
    if (g_arena) {
      p = static_cast<T*>(g_arena->take((int64_t)bytes));
      if (!p) raise(DBNET_ENOMEM, "request arena has no free range of " + std::to_string(bytes) + " bytes");
      ar = g_arena;
      n = count;
      return;
    }
    p = static_cast<T*>(dev_alloc(bytes, hk, hk_stream, "device state"));
    n = count;
  }
  void reset() {
    if (p) {
      if (ar) ar->give(p, (int64_t)(sizeof(T) * (size_t)n));
      else dev_free(p, sizeof(T) * (size_t)n, hk, hk_stream);
    }
    p = nullptr;
    n = 0;
    ar = nullptr;
  }
};

struct GraphDev {
  int32_t N = 0, R = 0;
  int64_t E = 0;
  std::vector<int32_t> ro_h, nexc_h;
  DevBuf<int64_t> row_ptr;
  DevBuf<uint16_t> rec;  // [3E] interleaved (target lo, target hi, BF16 weight),
                         // or [4E] with a second BF16 weight per edge
  DevBuf<int32_t> ro;
  DevBuf<uint8_t> seg;  // [N][seg_stride] u16 or u32 segment table
  int32_t seg_kind = 0, seg_stride = 0;
  bool packed = true;  // edges held as interleaved records
  bool rounded = false;
  bool two_w = false;  // a second weight per edge (8-byte records)
  int32_t max_delay = 1, kin_max = 0;
  double w_max = 0.0;
  // the smallest delay from which every delay carries fewer than
  // kEmitSegEdges edges per row on average (estimated on a sample of rows),
  // or 0 when there is none: those short segments are handed on at emission
  int32_t emit_from = 0;
};
constexpr double kEmitSegEdges = 4.0;

struct InstSpec {
  std::shared_ptr<GraphDev> graph;
  std::vector<dbnet_region_params_t> params;  // [R]
  dbnet_options_t opt;
  uint64_t net_id = 0;
};

struct InstHost {
  std::shared_ptr<GraphDev> graph;
  std::vector<RegionConst> rc_h;
  DevBuf<RegionConst> rc;
  DevBuf<double> bold;
  DevBuf<int32_t> raster_step, raster_id;
  InstDesc desc;
  dbnet_options_t opt;
  uint64_t net_id = 0;
  int32_t first_tile = 0, n_tiles = 0, rbase = 0;
  // host sources of the placement copies (kept until the instance goes)
  std::vector<int4> stage_ti;
  std::vector<int32_t> stage_ri;
  std::vector<double> stage_bw;
  std::vector<float> stage_fext;
  InstDyn stage_dyn{};
};

struct Engine {
  static constexpr int kChunk = 64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<InstHost> inst;
  DevBuf<float> V, J, Ibg, fext;
  DevBuf<uint8_t> ref;
  DevBuf<int2> acc;        // [acc_slots][stride] accumulators
  DevBuf<uint16_t> slot_emit;
  DevBuf<InstDesc> desc;
  DevBuf<InstDyn> dyn;
  DevBuf<int4> tile_info;
  DevBuf<int32_t> region_inst, cnt;
  DevBuf<long long> closed;
  DevBuf<double> bw, ylast;
  DevBuf<uint32_t> hist, hcount;
  DevBuf<uint16_t> hseg;
  DevBuf<int64_t> hr0;
  DevBuf<unsigned long long> base, events;  // base: the two graph-half iteration words
  DevBuf<unsigned> flags;
  unsigned long long g_host = 0;            // iterations enqueued so far
  EngineDev dev{};
  cudaGraphExec_t gexec = nullptr;
  int del_grid = 0;
  // launch-shape autotuner: from iteration tune_at on, one chunk per
  // candidate (delivery grid x sequential, pipelined or persistent
  // schedule), timed by CUDA events; the fastest stays
  static constexpr int kTuneRounds = 3;
  static constexpr double kDropped = 1e30;  // tune_ms of a candidate out of the running
  bool tune_pending = false;
  unsigned long long tune_at = 0;
  int tune_done = 0;                  // steps timed so far
  std::vector<int> tune_grid;         // candidates
  std::vector<double> tune_ms;        // chunk time per candidate (grid-major, schedule)
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  // pipelined schedule: the long part of step g + 1's delivery beside step
  // g's update on a second stream; long_pending: that part of step g_host is
  // already enqueued
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool pipelined = false;
  bool long_pending = false;
  int32_t fixed_schedule = 0;         // DBNET_SCHEDULE_*
  // persistent schedule: up to kPersistSteps steps per cooperative launch
  // of del_grid blocks (at most persist_max co-resident), pbar the grid
  // barrier's word; a barrier wait gives up after kBarrierLimitNs
  static constexpr int kPersistSteps = 4096;
  static constexpr unsigned long long kBarrierLimitNs = 1000000000ull;
  bool persistent = false;
  int persist_max = 0;
  bool persist_tunable = false;  // the tuner may weigh the persistent schedule
  DevBuf<unsigned> pbar;
  void direct_step();
  // sched: 0 sequential, 1 pipelined, 2 persistent
  void set_shape(int grid, int sched);
  void finish_turn(int n_candidates);
  // emission threshold: the engine's current d_emit (D + 1: none) and the
  // candidate the tuner weighs against "none" (0: no ring, nothing to tune).
  // Each candidate runs kEmitWarm + kEmitTimed steps (D of them for the
  // spikes in flight to pass), the last kEmitTimed timed as whole steps.
  static constexpr int kEmitTimed = 64;
  int32_t emit_cand = 0;
  int emit_phase = 0;                 // 0, 1: timing none / the candidate; 2: done
  int64_t emit_steps = 0;             // steps run in the current phase
  double emit_ms[2] = {0.0, 0.0};
  cudaEvent_t emit_ev[2] = {nullptr, nullptr};
  void set_emit(int32_t d);
  int32_t n_tiles = 0, total_R = 0, shift_S = 16;  // extents the kernels cover
  int64_t stride = 0;
  int32_t cap_tiles = 0, cap_R = 0, cap_inst = 0;    // capacities
  std::vector<int4> no_tiles_h;                       // copy sources that clear
  std::vector<InstDyn> zero_dyn_h;                    //   tiles and counters
  bool poisoned = false;
  std::string poison_msg;

  Engine() = default;
  Engine(const Engine&) = delete;
  ~Engine();
  // A fixed set of instances laid out end to end, sharing one fixed-point S.
  void init(const std::vector<InstSpec>& specs, void* user_stream);
  // Empty capacity for instances placed later: every tile and region slot
  // starts unused (the kernels skip it); D = longest delay + 1.
  // any_ext: launch the update variant with the OU current and the
  // per-neuron injected-current factors; four: four accumulator channels
  // per neuron, so that instances may carry two weights per edge.
  // emit_from: delays >= it may be handed on at emission (0: never; the
  // accumulators then have one slot).
  void init_pool(int32_t n_inst, int64_t tiles, int32_t regions, int32_t D,
                 const dbnet_options_t& common, void* user_stream, bool any_ext,
                 bool four = false, int32_t emit_from = 0);
  int64_t tune_emit(int64_t n);
  // Put instance k on tiles [first_tile, +tiles of its graph) and region
  // slots [rbase, +R): its constants, buffers and initial state; its step 0
  // is the next iteration enqueued, and it stops after n_end steps.
  void place(int k, const InstSpec& sp, int32_t first_tile, int32_t rbase, int S, long long n_end);
  // Mark instance k's tiles and region slots unused and drop its buffers.
  // The caller guarantees no enqueued kernel still reads them.
  void vacate(int k);
  // Tiles and region slots the kernels cover; a change re-captures the graph.
  void set_extent(int32_t tiles, int32_t regions);
  void check() const;
  void capture();
  void step(int64_t n);
  void run_plain(int64_t n);
  int64_t tune_steps(int64_t n);
  void step_timed(int64_t n, double* ms);
  void sync();
  InstDyn read_dyn(int k);
  int64_t bold_samples(int k) const;
};

std::shared_ptr<GraphDev> upload_graph(const dbnet_graph_t* g, cudaStream_t s);
// min_ref: the fewest refractory steps a region may have (spike binning)
void check_params(const dbnet_region_params_t& p, double dt, int32_t min_ref);
int32_t bin_lead(const dbnet_options_t& o);
void check_options(const dbnet_options_t& o);
RegionConst region_const(const dbnet_region_params_t& p, double dt, int S, int32_t start,
                         int32_t end, int32_t exc_end);

}  // namespace dbn

// A network handle: owns its engine, or views one instance of an ensemble.
struct dbnet {
  std::unique_ptr<dbn::Engine> own;  // null for a member view of an ensemble
  dbn::Engine* eng = nullptr;
  int inst = 0;
};

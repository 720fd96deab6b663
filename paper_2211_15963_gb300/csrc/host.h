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

// A sub-allocator over one device allocation (first fit, 256-byte granules,
// neighbours merged on release).  Used by the request server, so that
// admitting and retiring requests never calls cudaMalloc or cudaFree (the
// latter waits for the whole device).  Not thread-safe.
class Arena {
 public:
  Arena() = default;
  Arena(const Arena&) = delete;
  Arena& operator=(const Arena&) = delete;
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  void init(int64_t bytes) {
    bytes = round(bytes);
    cudaError_t e = cudaMalloc((void**)&base_, (size_t)bytes);
    if (e != cudaSuccess) {
      base_ = nullptr;
      cudaGetLastError();
      raise(e == cudaErrorMemoryAllocation ? DBNET_ENOMEM : DBNET_ECUDA,
            "cudaMalloc of the " + std::to_string(bytes) + "-byte request arena: " +
                cudaGetErrorString(e));
    }
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
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n), ar(o.ar) { o.p = nullptr; o.n = 0; o.ar = nullptr; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      reset();
      p = o.p; n = o.n; ar = o.ar;
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
    cudaError_t e = cudaMalloc((void**)&p, bytes);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      raise(e == cudaErrorMemoryAllocation ? DBNET_ENOMEM : DBNET_ECUDA,
            "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    n = count;
  }
  void reset() {
    if (p) {
      if (ar) ar->give(p, (int64_t)(sizeof(T) * (size_t)n));
      else cudaFree(p);
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
};

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
  DevBuf<int2> acc;
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
  // delivery-grid autotuner: from iteration tune_at on, kTuneRounds rounds
  // over the candidate grids, each step's delivery timed by CUDA events;
  // the fastest total wins and the step graph is captured again
  static constexpr int kTuneRounds = 16;
  bool tune_pending = false;
  unsigned long long tune_at = 0;
  int tune_done = 0;                  // steps timed so far
  std::vector<int> tune_grid;         // candidates
  std::vector<double> tune_ms;        // summed delivery time per candidate
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
  void init_pool(int32_t n_inst, int64_t tiles, int32_t regions, int32_t D,
                 const dbnet_options_t& common, void* user_stream, bool any_ext,
                 bool four = false);
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
void check_params(const dbnet_region_params_t& p, double dt);
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

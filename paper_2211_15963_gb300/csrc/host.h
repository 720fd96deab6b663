// Host-side engine types shared by engine.cu and ens.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "dbnet.h"
#include "engine.h"

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

// Device allocation owned by its holder.
template <class T>
struct DevBuf {
  T* p = nullptr;
  int64_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { reset(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { reset(); }
  void alloc(int64_t count) {
    reset();
    if (count <= 0) return;
    cudaError_t e = cudaMalloc((void**)&p, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      raise(e == cudaErrorMemoryAllocation ? DBNET_ENOMEM : DBNET_ECUDA,
            "cudaMalloc of " + std::to_string(sizeof(T) * (size_t)count) + " bytes: " +
                cudaGetErrorString(e));
    }
    n = count;
  }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

struct GraphDev {
  int32_t N = 0, R = 0;
  int64_t E = 0;
  std::vector<int32_t> ro_h, nexc_h;
  DevBuf<int64_t> row_ptr;
  DevBuf<uint16_t> rec;  // [3E] interleaved (target lo, target hi, BF16 weight)
  DevBuf<int32_t> ro;
  DevBuf<uint8_t> seg;  // [N][seg_stride] u16 or u32 segment table
  int32_t seg_kind = 0, seg_stride = 0;
  bool packed = true;  // edges held as interleaved records
  bool rounded = false;
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
};

struct Engine {
  static constexpr int kChunk = 64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<InstHost> inst;
  DevBuf<float> V, J;
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
  int32_t n_tiles = 0, total_R = 0, shift_S = 16;
  int64_t stride = 0;
  bool poisoned = false;
  std::string poison_msg;

  Engine() = default;
  Engine(const Engine&) = delete;
  ~Engine();
  void init(const std::vector<InstSpec>& specs, void* user_stream);
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

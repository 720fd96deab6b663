// Request server (dbsrv_* in dbnet.h): continuous batching of independent
// simulation requests on one engine.
//
// The engine is created empty with fixed capacities (init_pool): request
// slots, 1024-neuron tiles, region slots and a spike ring deep enough for
// the longest allowed delay.  A request occupies one slot, a contiguous run
// of tiles and of region slots, and arena memory for its graph, region
// constants and output buffers.  Every round enqueues chunk_steps steps of
// the whole engine (one update and one delivery launch per step for all
// resident requests, replayed from the engine's captured graph); each
// request's own step counter starts at its admission and stops at n_steps,
// after which its kernels leave it unchanged.
//
// Lifetime of a slot: RUNNING until the device has completed the request's
// last step (the host learns this from the event recorded after each
// round), then its results are copied out and it cools down for D more
// completed iterations -- until then a spike it emitted may still be
// delivered, which reads its edge records -- and only then are its tiles,
// region slots and memory reused.  Graph uploads run on a second stream,
// so the rounds already enqueued keep the device busy meanwhile.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "dbnet.h"
#include "engine.h"
#include "host.h"

namespace dbn {
int choose_shift(const GraphDev& g, double wext_max, int32_t requested);

namespace {

double now_s() {
  using clk = std::chrono::steady_clock;
  return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

struct Req {
  int64_t id = 0;
  dbnet_graph_t graph{};                       // caller's host arrays (until admitted)
  std::vector<dbnet_region_params_t> params;
  dbsrv_request_t rq{};
  int32_t state = DBSRV_QUEUED;
  int32_t error = 0;
  std::string msg;
  int32_t slot = -1, first_tile = 0, n_tiles = 0, rbase = 0, R = 0;
  unsigned long long g0 = 0, g_end = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int64_t spikes = 0;
  std::vector<double> bold;                    // [n][R]
  int64_t n_bold = 0;
  std::vector<int32_t> r_step, r_id;           // sorted by (step, id)
};

struct Slot {
  int64_t req = -1;                 // request using it, -1 when free
  bool cooling = false;
  unsigned long long free_at = 0;   // completed iteration at which it may be reused
};

struct Round {
  unsigned long long g_after;
  cudaEvent_t ev;
};

}  // namespace
}  // namespace dbn

struct dbsrv {
  std::unique_ptr<dbn::Engine> eng;
  dbsrv_options_t opt{};
  dbn::Arena arena;
  cudaStream_t up = nullptr;  // graph uploads and result reads
  std::map<int64_t, std::unique_ptr<dbn::Req>> reqs;
  std::deque<int64_t> queue;
  std::vector<dbn::Slot> slots;
  dbn::FreeList<int32_t> tiles, regions;  // first fit over tiles and region slots
  std::map<uint64_t, std::weak_ptr<dbn::GraphDev>> shared;
  std::deque<dbn::Round> rounds;
  std::vector<cudaEvent_t> spare;
  unsigned long long g_done = 0;
  int64_t next_id = 1;
  int32_t n_done = 0;
  bool poisoned = false;
  std::string poison_msg;

  ~dbsrv() {
    if (eng && eng->stream) cudaStreamSynchronize(eng->stream);
    for (auto& r : rounds) cudaEventDestroy(r.ev);
    for (auto e : spare) cudaEventDestroy(e);
    reqs.clear();
    eng.reset();  // instances release their arena ranges first
    if (up) cudaStreamDestroy(up);
  }
};

namespace dbn {
namespace {

constexpr int kAdmitScan = 8;  // queued requests looked at per round

template <class F>
int srv_guard(dbsrv* s, F&& f) {
  if (s && s->poisoned) {
    g_last_error = "server poisoned by an earlier failure: " + s->poison_msg;
    return DBNET_ESTATE;
  }
  try {
    f();
    return DBNET_OK;
  } catch (const Error& e) {
    g_last_error = e.msg;
    if (s && e.code == DBNET_ECUDA) {
      s->poisoned = true;
      s->poison_msg = e.msg;
    }
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return DBNET_ENOMEM;
  } catch (...) {
    g_last_error = "unexpected exception";
    return DBNET_ECUDA;
  }
}

int32_t tiles_for(int32_t N) { return (N + kTile - 1) / kTile; }

// Device bytes a request needs from the arena when its graph is not shared:
// records, row pointers, segment table, staging, region constants, BOLD,
// raster (rounded up generously; admission still handles a failed take).
int64_t arena_estimate(const Req& r, int32_t dmax) {
  const dbnet_graph_t& g = r.graph;
  const int64_t N = g.n_neurons, E = g.row_ptr[N], R = g.n_regions;
  const int64_t stride = (dmax + 7) / 8 * 8;
  const bool two = g.weight2 != nullptr;
  const int64_t stage = std::min<int64_t>(E, int64_t(1) << 27) * (two ? 13 : 9);
  return (two ? 8 : 6) * E + 8 * (N + 1) + 4 * stride * N + stage + 8 * N + 4 * (R + 1) +
         (int64_t)sizeof(RegionConst) * R + 8 * std::max<int64_t>(r.rq.bold_capacity, 1) * R +
         8 * r.rq.raster_capacity + (int64_t(1) << 20);
}

void poll_rounds(dbsrv* s) {
  while (!s->rounds.empty()) {
    const cudaError_t q = cudaEventQuery(s->rounds.front().ev);
    if (q == cudaErrorNotReady) break;
    CK(q);
    s->g_done = s->rounds.front().g_after;
    s->spare.push_back(s->rounds.front().ev);
    s->rounds.pop_front();
  }
}

void wait_oldest(dbsrv* s) {
  if (s->rounds.empty()) return;
  CK(cudaEventSynchronize(s->rounds.front().ev));
  poll_rounds(s);
}

// Copy a finished request's results to the host; its slot starts cooling.
void complete(dbsrv* s, Req& r) {
  Engine& e = *s->eng;
  const InstHost& ih = e.inst[(size_t)r.slot];
  InstDyn d;
  CK(cudaMemcpyAsync(&d, e.dyn.p + r.slot, sizeof(d), cudaMemcpyDeviceToHost, s->up));
  const int64_t samples = r.rq.n_steps / ih.desc.spb / ih.desc.bins_per_tr;
  r.n_bold = std::min<int64_t>(samples, ih.opt.bold_capacity);
  r.bold.assign((size_t)(r.n_bold * r.R), 0.0);
  if (r.n_bold > 0)
    CK(cudaMemcpyAsync(r.bold.data(), ih.bold.p, sizeof(double) * r.n_bold * r.R,
                       cudaMemcpyDeviceToHost, s->up));
  CK(cudaStreamSynchronize(s->up));
  r.spikes = (int64_t)d.spikes;
  const int64_t n = std::min<int64_t>((int64_t)d.raster_count, ih.opt.raster_capacity);
  if (n > 0) {
    std::vector<int32_t> st((size_t)n), id((size_t)n);
    CK(cudaMemcpyAsync(st.data(), ih.raster_step.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->up));
    CK(cudaMemcpyAsync(id.data(), ih.raster_id.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->up));
    CK(cudaStreamSynchronize(s->up));
    std::vector<uint64_t> key((size_t)n);
    for (int64_t k = 0; k < n; ++k)
      key[(size_t)k] = ((uint64_t)(uint32_t)st[(size_t)k] << 32) | (uint32_t)id[(size_t)k];
    std::sort(key.begin(), key.end());
    r.r_step.resize((size_t)n);
    r.r_id.resize((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
      r.r_step[(size_t)k] = (int32_t)(key[(size_t)k] >> 32);
      r.r_id[(size_t)k] = (int32_t)(key[(size_t)k] & 0xFFFFFFFFu);
    }
  }
  r.state = DBSRV_DONE;
  r.t_done = now_s();
  ++s->n_done;
  Slot& sl = s->slots[(size_t)r.slot];
  sl.cooling = true;
  sl.free_at = r.g_end + (unsigned long long)e.dev.D;
}

void release_slot(dbsrv* s, int k) {
  Slot& sl = s->slots[(size_t)k];
  Engine& e = *s->eng;
  const InstHost& ih = e.inst[(size_t)k];
  if (ih.graph) {
    s->tiles.give(ih.first_tile, ih.n_tiles);
    s->regions.give(ih.rbase, ih.graph->R);
  }
  e.vacate(k);
  sl = Slot{};
}

// Highest tile and region slot in use (running or cooling), plus one.
void fit_extent(dbsrv* s) {
  Engine& e = *s->eng;
  int32_t t = 0, r = 0;
  for (size_t k = 0; k < s->slots.size(); ++k) {
    if (s->slots[k].req < 0) continue;
    const InstHost& ih = e.inst[k];
    t = std::max(t, ih.first_tile + ih.n_tiles);
    r = std::max(r, ih.rbase + ih.graph->R);
  }
  // grow at once; shrink only by a quarter or more (each change re-captures)
  if (t > e.n_tiles || r > e.total_R || t < e.n_tiles * 3 / 4 || r < e.total_R * 3 / 4)
    e.set_extent(std::max(t, 1), std::max(r, 1));
}

// Try to admit request r now.  Returns false when it does not fit yet.
bool admit(dbsrv* s, Req& r) {
  Engine& e = *s->eng;
  int k = -1;
  for (size_t i = 0; i < s->slots.size(); ++i)
    if (s->slots[i].req < 0) {
      k = (int)i;
      break;
    }
  if (k < 0) return false;
  const int32_t nt = tiles_for(r.graph.n_neurons);
  if (!s->tiles.fits(nt) || !s->regions.fits(r.graph.n_regions)) return false;
  std::shared_ptr<GraphDev> gd;
  if (r.rq.graph_key) {
    auto it = s->shared.find(r.rq.graph_key);
    if (it != s->shared.end()) gd = it->second.lock();
  }
  if (!gd && arena_estimate(r, s->opt.max_delay) > s->arena.largest_free()) return false;
  const int32_t t0 = s->tiles.take(nt);
  const int32_t r0 = s->regions.take(r.graph.n_regions);
  try {
    ArenaScope scope(&s->arena);
    if (!gd) {
      gd = upload_graph(&r.graph, s->up);
      if (r.rq.graph_key) s->shared[r.rq.graph_key] = gd;
    }
    double wext_max = 0.0;
    for (const auto& p : r.params) wext_max = std::max(wext_max, p.w_ext);
    const int S = choose_shift(*gd, wext_max, s->opt.run.fixed_shift);
    InstSpec sp;
    sp.graph = gd;
    sp.params = r.params;
    sp.opt = s->opt.run;
    sp.opt.seed = r.rq.seed;
    sp.opt.net_id = r.rq.net_id;
    sp.opt.raster_capacity = r.rq.raster_capacity;
    sp.opt.bold_capacity = r.rq.bold_capacity;
    sp.net_id = r.rq.net_id;
    e.place(k, sp, t0, r0, S, (long long)r.rq.n_steps);
  } catch (const Error& err) {
    s->tiles.give(t0, nt);
    s->regions.give(r0, r.graph.n_regions);
    if (err.code == DBNET_ENOMEM) return false;  // the arena is fragmented: wait
    if (err.code == DBNET_ECUDA) throw;
    r.state = DBSRV_FAILED;
    r.error = err.code;
    r.msg = err.msg;
    r.t_done = now_s();
    return true;
  }
  r.slot = k;
  r.first_tile = t0;
  r.n_tiles = nt;
  r.rbase = r0;
  r.R = r.graph.n_regions;
  r.g0 = e.g_host;
  r.g_end = r.g0 + (unsigned long long)r.rq.n_steps;
  r.state = DBSRV_RUNNING;
  r.t_admit = now_s();
  r.graph = dbnet_graph_t{};  // the caller's arrays are no longer needed
  s->slots[(size_t)k].req = r.id;
  return true;
}

void pump(dbsrv* s) {
  Engine& e = *s->eng;
  e.check();
  poll_rounds(s);
  // results of requests whose last step has completed
  for (auto& sl : s->slots) {
    if (sl.req < 0 || sl.cooling) continue;
    Req& r = *s->reqs.at(sl.req);
    if (r.g_end <= s->g_done) complete(s, r);
  }
  // slots whose spikes can no longer be in flight
  for (size_t k = 0; k < s->slots.size(); ++k)
    if (s->slots[k].req >= 0 && s->slots[k].cooling && s->slots[k].free_at <= s->g_done)
      release_slot(s, (int)k);
  // admission: first fit over the oldest queued requests
  int scanned = 0;
  for (auto it = s->queue.begin(); it != s->queue.end() && scanned < kAdmitScan;) {
    ++scanned;
    Req& r = *s->reqs.at(*it);
    if (admit(s, r)) it = s->queue.erase(it);
    else ++it;
  }
  bool busy = false;
  for (const auto& sl : s->slots) busy = busy || sl.req >= 0;
  if (!busy) {
    // an empty pool that cannot take the oldest request never will
    if (!s->queue.empty()) {
      Req& r = *s->reqs.at(s->queue.front());
      r.state = DBSRV_FAILED;
      r.error = DBNET_ERANGE;
      r.msg = "the request does not fit the empty pool (arena or tiles)";
      r.t_done = now_s();
      s->queue.pop_front();
    }
    return;
  }
  fit_extent(s);
  // one round for every resident request
  if ((int)s->rounds.size() >= s->opt.max_inflight) wait_oldest(s);
  e.step(s->opt.chunk_steps);
  cudaEvent_t ev;
  if (!s->spare.empty()) {
    ev = s->spare.back();
    s->spare.pop_back();
  } else {
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  }
  CK(cudaEventRecord(ev, e.stream));
  s->rounds.push_back(Round{e.g_host, ev});
}

void fill_stats(dbsrv* s, dbsrv_stats_t* out) {
  std::memset(out, 0, sizeof(*out));
  Engine& e = *s->eng;
  unsigned long long ev = 0;
  CK(cudaMemcpyAsync(&ev, e.events.p, sizeof(ev), cudaMemcpyDeviceToHost, s->up));
  CK(cudaStreamSynchronize(s->up));
  out->iterations = (int64_t)s->g_done;
  out->events = (int64_t)ev;  // counted at each spike's delay-1 delivery
  for (const auto& sl : s->slots) {
    if (sl.req < 0) continue;
    if (sl.cooling) ++out->cooling;
    else ++out->running;
  }
  out->queued = (int32_t)s->queue.size();
  out->done = s->n_done;
  out->arena_used = s->arena.used();
  out->arena_bytes = s->arena.size();
  int32_t used = 0;
  for (size_t k = 0; k < s->slots.size(); ++k)
    if (s->slots[k].req >= 0) used += e.inst[k].n_tiles;
  out->tiles_in_use = used;
  out->tile_extent = e.n_tiles;
}

}  // namespace
}  // namespace dbn

using namespace dbn;

extern "C" {

int dbsrv_options_default(dbsrv_options_t* o) {
  if (!o) return DBNET_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->max_neurons = int64_t(8) << 20;
  o->max_requests = 64;
  o->max_regions = 1024;
  o->max_delay = 255;
  o->chunk_steps = 256;
  o->arena_bytes = int64_t(64) << 30;
  o->max_inflight = 2;
  return dbnet_options_default(&o->run);
}

int dbsrv_create(const dbsrv_options_t* options, void* cuda_stream, dbsrv_t** out) {
  if (!options || !out) return DBNET_EINVAL;
  *out = nullptr;
  auto s = std::make_unique<dbsrv>();
  int rc = srv_guard(nullptr, [&] {
    AllocStreamScope alloc_stream(cuda_stream);
    const dbsrv_options_t& o = *options;
    check_options(o.run);
    if (o.max_neurons < 1 || o.max_requests < 1 || o.max_regions < 1 || o.chunk_steps < 1 ||
        o.max_inflight < 1 || o.arena_bytes < (int64_t(1) << 20))
      raise(DBNET_EINVAL, "server capacities must be positive (arena >= 1 MiB)");
    if (o.max_delay < 1 || o.max_delay > 255) raise(DBNET_EINVAL, "max_delay must be 1..255");
    if (o.two_weights != 0 && o.two_weights != 1) raise(DBNET_EINVAL, "two_weights must be 0 or 1");
    const int64_t tiles = (o.max_neurons + kTile - 1) / kTile;
    if (tiles * kTile >= (int64_t(1) << 31)) raise(DBNET_EINVAL, "max_neurons too large");
    s->opt = o;
    s->eng.reset(new Engine());
    s->eng->init_pool(o.max_requests, tiles, o.max_regions, o.max_delay + 1 + bin_lead(o.run), o.run, cuda_stream,
                      true,  // any request may bring the OU current
                      o.two_weights != 0);
    s->eng->set_extent(1, 1);
    s->arena.init(o.arena_bytes);
    CK(cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking));
    s->slots.assign((size_t)o.max_requests, Slot{});
    s->tiles.reset((int32_t)tiles);
    s->regions.reset(o.max_regions);
    CK(cudaStreamSynchronize(s->eng->stream));
  });
  if (rc == DBNET_OK) *out = s.release();
  return rc;
}

int dbsrv_submit(dbsrv_t* s, const dbnet_graph_t* graph, const dbnet_region_params_t* params,
                 const dbsrv_request_t* request, int64_t* id) {
  if (!s || !graph || !params || !request || !id) return DBNET_EINVAL;
  return srv_guard(s, [&] {
    const dbnet_graph_t& g = *graph;
    const int32_t N = g.n_neurons, R = g.n_regions;
    if (N < 1 || R < 1 || !g.region_offsets || !g.n_exc || !g.row_ptr)
      raise(DBNET_EINVAL, "malformed graph");
    if (request->n_steps < 1) raise(DBNET_EINVAL, "n_steps must be >= 1");
    if (request->bold_capacity < 0 || request->raster_capacity < 0)
      raise(DBNET_EINVAL, "negative capacity");
    if ((int64_t)tiles_for(N) > s->eng->cap_tiles || R > s->eng->cap_R)
      raise(DBNET_ERANGE, "the request is larger than the server's pool");
    if (g.weight2 && !s->opt.two_weights)
      raise(DBNET_EUNSUPPORTED, "two weights per edge need a server created with two_weights = 1");
    for (int32_t r = 0; r < R; ++r) check_params(params[r], s->opt.run.dt_ms, bin_lead(s->opt.run));
    auto q = std::make_unique<Req>();
    q->id = s->next_id++;
    q->graph = g;
    q->params.assign(params, params + R);
    q->rq = *request;
    if (q->rq.bold_capacity == 0) {
      const int64_t spb = std::lrint(s->opt.run.bin_ms / s->opt.run.dt_ms);
      const int64_t bpt = std::lrint(s->opt.run.tr_ms / s->opt.run.bin_ms);
      q->rq.bold_capacity = std::max<int64_t>(1, request->n_steps / spb / bpt);
    }
    q->t_submit = now_s();
    *id = q->id;
    s->queue.push_back(q->id);
    s->reqs[q->id] = std::move(q);
  });
}

int dbsrv_pump(dbsrv_t* s, dbsrv_stats_t* out) {
  if (!s) return DBNET_EINVAL;
  return srv_guard(s, [&] {
    pump(s);
    if (out) fill_stats(s, out);
  });
}

int dbsrv_drain(dbsrv_t* s) {
  if (!s) return DBNET_EINVAL;
  return srv_guard(s, [&] {
    for (;;) {
      bool busy = !s->queue.empty();
      for (const auto& sl : s->slots) busy = busy || sl.req >= 0;
      if (!busy) break;
      pump(s);
    }
    CK(cudaStreamSynchronize(s->eng->stream));
    poll_rounds(s);
  });
}

int dbsrv_poll(dbsrv_t* s, int64_t id, dbsrv_status_t* out) {
  if (!s || !out) return DBNET_EINVAL;
  return srv_guard(s, [&] {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) raise(DBNET_EINVAL, "unknown request id");
    const Req& r = *it->second;
    std::memset(out, 0, sizeof(*out));
    out->state = r.state;
    out->error = r.error;
    if (r.state == DBSRV_RUNNING)
      out->steps = (int64_t)std::min<unsigned long long>(
          s->g_done > r.g0 ? s->g_done - r.g0 : 0ull, (unsigned long long)r.rq.n_steps);
    else if (r.state == DBSRV_DONE)
      out->steps = r.rq.n_steps;
    out->spikes = r.spikes;
    out->bold_samples = r.n_bold;
    out->raster_len = (int64_t)r.r_step.size();
    const double t_now = now_s();
    const double t_adm = r.state == DBSRV_QUEUED ? t_now : (r.t_admit > 0 ? r.t_admit : r.t_done);
    out->queued_s = t_adm - r.t_submit;
    const double t_end = (r.state == DBSRV_DONE || r.state == DBSRV_FAILED) ? r.t_done : t_now;
    out->run_s = r.state == DBSRV_QUEUED ? 0.0 : t_end - t_adm;
    out->latency_s = t_end - r.t_submit;
    if (r.state == DBSRV_FAILED) g_last_error = r.msg;
  });
}

int dbsrv_read_bold(dbsrv_t* s, int64_t id, double* y, int64_t cap_samples, int64_t* n_out) {
  if (!s || !n_out || cap_samples < 0 || (cap_samples > 0 && !y)) return DBNET_EINVAL;
  *n_out = 0;
  return srv_guard(s, [&] {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) raise(DBNET_EINVAL, "unknown request id");
    const Req& r = *it->second;
    if (r.state != DBSRV_DONE) raise(DBNET_ESTATE, "the request has no results yet");
    if (r.n_bold > cap_samples) raise(DBNET_ERANGE, "cap_samples is too small");
    std::copy(r.bold.begin(), r.bold.end(), y);
    *n_out = r.n_bold;
  });
}

int dbsrv_read_spikes(dbsrv_t* s, int64_t id, int32_t* step, int32_t* nid, int64_t cap,
                      int64_t* n_out) {
  if (!s || !n_out || cap < 0 || (cap > 0 && (!step || !nid))) return DBNET_EINVAL;
  *n_out = 0;
  return srv_guard(s, [&] {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) raise(DBNET_EINVAL, "unknown request id");
    const Req& r = *it->second;
    if (r.state != DBSRV_DONE) raise(DBNET_ESTATE, "the request has no results yet");
    const int64_t n = (int64_t)r.r_step.size();
    if (n > cap) raise(DBNET_ERANGE, "cap is too small");
    std::copy(r.r_step.begin(), r.r_step.end(), step);
    std::copy(r.r_id.begin(), r.r_id.end(), nid);
    *n_out = n;
  });
}

int dbsrv_release(dbsrv_t* s, int64_t id) {
  if (!s) return DBNET_EINVAL;
  return srv_guard(s, [&] {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) raise(DBNET_EINVAL, "unknown request id");
    Req& r = *it->second;
    if (r.state == DBSRV_RUNNING) raise(DBNET_ESTATE, "the request is running");
    if (r.state == DBSRV_QUEUED) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), id));
    if (r.state == DBSRV_DONE) --s->n_done;
    s->reqs.erase(it);
  });
}

int dbsrv_stats(dbsrv_t* s, dbsrv_stats_t* out) {
  if (!s || !out) return DBNET_EINVAL;
  return srv_guard(s, [&] { fill_stats(s, out); });
}

void dbsrv_destroy(dbsrv_t* s) { delete s; }

}  // extern "C"

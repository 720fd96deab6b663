// Device data layout shared by the kernels and the host engine.
//
// One engine steps a set of instances (networks) together.  A single network
// is an engine with one instance; an HMDA ensemble is an engine whose
// instances share one graph and differ in their region constants and Philox
// key.  Global neuron index space: instance k occupies
// [base_k, base_k + N_k), base_k a multiple of kTile, so every update block
// (one tile) belongs to exactly one instance.
//
// HBM layout (per global neuron i, stride = padded neuron count):
//   V[i] f32 | J[u * stride + i] f32, u = AMPA, NMDA, GABA_A, GABA_B |
//   ref[i] u8 (remaining refractory steps) | acc[i] int2 (E, I fixed point)
// Edges of an instance (CSR by source, rows sorted by delay):
//   col[e] u32 = target | delay << shift  (or target, with delay[e] u8)
//   w[e]   u16 BF16 bit pattern
// Live delivery list: one 16-byte entry per spike whose later-delay edges are
// still to be delivered (position in the row, current delay, class, rows left,
// instance).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dbn {

constexpr int kTile = 1024;         // neurons per update block
constexpr int kUpdThreads = 256;    // four neurons per thread
constexpr int kDelThreads = 256;
constexpr int kMaxThr = 16;         // Poisson inversion thresholds

struct RegionConst {
  float dtC, gL, VL, Vth, Vreset, Iext;
  float g[4], Vu[4], dec[4];
  int32_t n_ref, q_ext, n_thr, exc_end;  // exc_end: first inhibitory local index
  int32_t start, end, pad0, pad1;        // local neuron range [start, end)
  uint32_t thr[kMaxThr];
};

struct InstDesc {
  const int64_t* row_ptr;
  const uint32_t* col;
  const uint16_t* w;
  const uint8_t* delay;          // nullptr when the delay is packed into col
  const int32_t* region_offsets; // [R+1], local
  const RegionConst* rc;         // [R]
  double* bold;                  // [bold_cap][R]
  int32_t* raster_step;
  int32_t* raster_id;
  int64_t base;
  int64_t raster_cap;
  int64_t bold_cap;
  uint64_t seed, net_id;
  int32_t N, R, rbase, shift;
  uint32_t tmask;
  float two_S, inv_two_S;
  int32_t spb, bins_per_tr;
  int32_t pad;
  double h_bw, z_scale, kappa, gamma, tau, alpha, rho, V0;
};

struct InstDyn {
  long long step;
  long long bins_done;
  long long bold_count;
  unsigned long long raster_count;
  unsigned long long spikes;
  int32_t active;
  int32_t pad;
};

struct __align__(16) Entry {
  unsigned long long pdc;  // position (48 bits) | delay done (8) | class (8)
  uint32_t rem;            // edges of the row not yet delivered
  uint32_t inst;
};

enum : unsigned {
  kFlagListOverflow = 1u,
  kFlagBoldOverflow = 2u,
};

struct EngineDev {
  float* V;
  float* J;
  uint8_t* ref;
  int2* acc;
  int64_t stride;
  const InstDesc* insts;
  InstDyn* dyn;
  const int32_t* tile_inst;
  int32_t* cnt;          // [total_R] spikes in the current bin
  double* bw;            // [total_R][4]
  double* ylast;         // [total_R]
  const int32_t* region_inst;
  Entry* list0;
  Entry* list1;
  uint32_t* count;       // [2]
  unsigned long long* iter;
  unsigned int* done;
  unsigned long long* events;
  unsigned int* flags;
  uint64_t list_cap;
  int32_t n_inst, n_tiles, total_R, pad;
};

// Launchers (kernels.cu)
void launch_init_state(const EngineDev& e, int inst, int n_tiles_inst, int first_tile,
                       cudaStream_t s);
void launch_update(const EngineDev& e, cudaStream_t s);
void launch_deliver(const EngineDev& e, int grid, cudaStream_t s);
int deliver_grid();
void launch_validate_pack(int32_t N, const int64_t* row_ptr, uint32_t* col, const void* w_in,
                          int32_t w_dtype, uint16_t* w_out, const uint8_t* delay_in,
                          int32_t shift, int32_t* indeg, unsigned* wmax_bits,
                          unsigned* dmax, unsigned* err, cudaStream_t s);
void launch_max_reduce(const int32_t* a, int64_t n, unsigned* out, cudaStream_t s);

enum : unsigned {
  kErrTarget = 1u,
  kErrDelayRange = 2u,
  kErrDelayOrder = 4u,
  kErrWeight = 8u,
  kErrRounded = 16u,
};

}  // namespace dbn

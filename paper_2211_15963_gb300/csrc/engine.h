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
//   ref[i] u8 (remaining refractory steps) | acc[i] int2 (E, I fixed point),
//   or, in an engine with four channels, acc[2i], acc[2i+1] (AMPA, NMDA |
//   GABA_A, GABA_B: one int4 per neuron)
// Edges of an instance (CSR by source, rows sorted by delay), either
//   rec[3e], rec[3e+1], rec[3e+2] u16 = target low, target high, BF16 weight
//     (interleaved 6-byte records: a short segment is one contiguous read), or,
//   with two weights per edge, rec[4e .. 4e+3] u16 = target low, target high,
//     BF16 weight, BF16 second weight (8-byte records, one load each), or,
//   for graphs the caller keeps (the allocation-free entry point), arrays
//   col[e] u32 = target, w[e] u16 BF16 bit pattern, delay[e] u8
//   seg[j * seg_stride + k] u16/u32 = number of edges of row j with
//                       delay <= k + 1, k < dmax (the per-delay segment
//                       table; seg_stride pads rows to 16 bytes)
// Iteration g of an engine runs k_deliver then k_update; the bin that ends
// with iteration g - 1 is closed (Balloon-Windkessel step, BOLD sample) at
// the start of k_deliver(g), one region per thread.
// Spike ring: D slots; slot n mod D lists the spikes handed on at step n
//   (their own step, or the last step of their bin with spike binning) as
//   global index | class << 31, with a count per slot.  At step n the
//   delivery reads slots n - d (d = 1..D-1) and applies, for each listed
//   spike, the segment of its row whose delay is exactly d (arrival time).
// Long delays at emission: when d_emit <= the longest delay, the
//   accumulators form a ring of D slots (slot a mod D collects the arrivals
//   of step a); at step n the delivery adds, for every spike handed on at
//   step n - 1, its edges of delay d >= d_emit straight into slot n - 1 + d,
//   each (spike, delay) segment read as it lies in the row, so that the
//   short segments of long delays cost one coalesced pass instead of one
//   resolution each; arrival time keeps the delays below d_emit.  The
//   update of step n reads and clears slot n.
// Delay-major segment ring (u16 tables only): k_deliver(n) copies, for the
//   first seg_cap spikes of step n - 1, the row start into hr0[slot][k] and
//   the row's segment counts into hseg[slot][d][k] (d < dcap), so that the
//   items (spike k, delay d) of later steps resolve with coalesced loads.
//   Spikes beyond seg_cap, delay-1 items and u32 tables read the graph's
//   own row_ptr and segment table instead.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace dbn {

// Philox4x64-10 (Salmon et al., SC'11): ten rounds, two 64x64->128 products
// per round with the published multipliers; the key advances by the Weyl
// constants after each round.  Host and device (the host draws the
// per-neuron injected-current factors at create).
__host__ __device__ __forceinline__ unsigned long long mulhi64(unsigned long long a,
                                                               unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
#endif
}
__host__ __device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                                       unsigned long long k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    unsigned long long hi0 = mulhi64(m0, c[0]), lo0 = m0 * c[0];
    unsigned long long hi1 = mulhi64(m1, c[2]), lo1 = m1 * c[2];
    unsigned long long n0 = hi1 ^ c[1] ^ k0;
    unsigned long long n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}

constexpr int kTile = 1024;         // neurons per update block
constexpr int kUpdThreads = 256;    // four neurons per thread
constexpr int kDelThreads = 256;
constexpr int kMaxThr = 16;         // Poisson inversion thresholds
constexpr int kTileRegions = 8;     // region constants staged in shared memory

// 16-byte multiples: the update kernel moves these with bulk copies
// (laid out as 16-byte vectors: the update kernel reads them with 128-bit loads)
struct alignas(16) RegionConst {
  float g[4];                        // channel conductance scales
  float Vu[4];                       // reversal potentials
  float dec[4];                      // per-step trace decay exp(-dt/tau_u)
  float dtC, gL, VL, Vth;
  float Vreset, Iext;
  int32_t n_ref, q_ext;
  int32_t n_thr, exc_end, start, end;  // exc_end: first inhibitory local index;
                                       // local neuron range [start, end)
  uint32_t thr[kMaxThr];             // Poisson inversion thresholds, non-decreasing
  float ou_mu, ou_k, ou_s;           // background OU current: mu, dt/tau,
  int32_t ext;                       //   sigma sqrt(2 dt/tau); kExt* bits
};
enum : int32_t {
  kExtOU = 1,    // background OU current
  kExtHet = 2,   // per-neuron injected-current factor
};

enum : int32_t {
  kSegSearch = 0,  // no table: binary search over the row's delays
  kSeg16 = 1,
  kSeg32 = 2,
};

struct alignas(16) InstDesc {
  const int64_t* row_ptr;
  const uint16_t* rec;           // interleaved records, or nullptr for col/w/delay
  const uint32_t* col;
  const uint16_t* w;
  const uint8_t* delay;          // col/w/delay: caller-held arrays (allocation-free runs)
  const void* seg;               // [N][seg_stride] segment table, or nullptr
  const int32_t* region_offsets; // [R+1], local
  const RegionConst* rc;         // [R]
  double* bold;                  // [bold_cap][R]
  int32_t* raster_step;
  int32_t* raster_id;
  int64_t base;
  int64_t raster_cap;
  int64_t bold_cap;
  uint64_t seed, net_id;
  unsigned long long g0;         // engine iteration at which this instance's step 0 ran
  long long n_end;               // steps it runs: later iterations leave it unchanged
  int32_t N, R, rbase, shift;    // shift, tmask: the col/w/delay form (targets col & tmask)
  uint32_t tmask;
  float two_S, inv_two_S;
  int32_t spb, bins_per_tr;
  int32_t seg_kind, dmax, seg_stride, ext;  // ext: kExt* bits of any region
  int32_t two_w, bin_sp;         // two_w: 8-byte records with a second weight; bin_sp:
                                 //   spikes handed on at the end of their bin
  double h_bw, z_scale, kappa, gamma, tau, alpha, rho, V0;
};

struct InstDyn {
  unsigned long long raster_count;
  unsigned long long spikes;
  int32_t active;
  int32_t pad;
};

// Where a kernel finds its engine iteration g: *base + off, or off when base
// is null (direct launches).  When next is set, the kernel also writes g + 1
// there (every block writes the same value), which lets a captured graph
// chain its halves through two base words.
struct StepRef {
  const unsigned long long* base;
  unsigned long long off;
  unsigned long long* next;
};

enum : unsigned {
  kFlagHistOverflow = 1u,  // a spike did not fit its ring slot (cannot happen: a slot holds every neuron)
  kFlagTimeout = 2u,       // a grid barrier of the persistent stepper gave up waiting
};

struct EngineDev {
  float* V;
  float* J;
  float* Ibg;            // background OU current per neuron
  float* fext;           // per-neuron injected-current factor (1 where homogeneous)
  uint8_t* ref;
  int2* acc;             // [acc_slots][stride] (int2, or int4 with four channels)
  int64_t stride;
  int32_t acc_slots;     // 1, or D when long delays are handed on at emission
  int32_t d_emit;        // delays >= d_emit are added at emission into the slot
                         //   of their arrival step (D + 1: none)
  uint16_t* slot_emit;   // [D] d_emit in force when each ring slot's spikes were
                         //   handed on (their delays below it arrive later)
  const InstDesc* insts;
  InstDyn* dyn;
  const int4* tile_info;  // per tile: instance, first region (local), regions touched, 0
  int32_t* cnt;          // [total_R] spikes in the current bin
  double* bw;            // [total_R][4]
  double* ylast;         // [total_R]
  const int32_t* region_inst;
  long long* closed;     // [total_R] last iteration whose bin was closed
  uint32_t* hist;        // [D][hist_cap]
  uint32_t* hcount;      // [D]
  int64_t hist_cap;
  uint16_t* hseg;        // [D][dcap][seg_cap]
  int64_t* hr0;          // [D][seg_cap]
  int64_t seg_cap;       // 0: no segment ring
  int32_t dcap;
  int32_t bin_lead;      // spike binning: steps per bin - 1 (else 0)
  unsigned long long* events;
  unsigned int* flags;
  int32_t D;
  int32_t n_inst, n_tiles, total_R;
  int32_t any_ext;       // launch the update variant with the kExt* terms
  int32_t phases;        // rank phases of the delivery's arrival items (1..8)
  int32_t four;          // four accumulator channels per neuron (acc as int4)
};

// Launchers (kernels.cu)
void launch_init_state(const EngineDev& e, int inst, int n_tiles_inst, int first_tile,
                       cudaStream_t s);
void launch_update(const EngineDev& e, StepRef sr, cudaStream_t s);
enum : int { kPartAll = 0, kPartLong = 1, kPartShort = 2 };  // see k_deliver
void launch_deliver(const EngineDev& e, int grid, StepRef sr, cudaStream_t s, int part = kPartAll);
// closes the bin that ends with iteration g - 1 (if any) for every region
void launch_close(const EngineDev& e, unsigned long long g, cudaStream_t s);
void launch_set_base(unsigned long long* base, unsigned long long g, cudaStream_t s);
int deliver_grid();
// The persistent stepper: iterations g0 .. g0 + nsteps - 1 (every part of
// the delivery, then the update, per iteration) in one cooperative launch
// of grid blocks, which must not exceed persist_max_grid(e) (0: the
// occupancy query failed).  *count is the grid barrier's word, cleared on s
// before the launch; each barrier wait gives up after limit_ns and sets
// kFlagTimeout in e.flags.  Returns the launch's error code.
int persist_max_grid(const EngineDev& e);
cudaError_t launch_persist(const EngineDev& e, int grid, unsigned long long g0, int nsteps,
                           unsigned* count, unsigned long long limit_ns, cudaStream_t s);
// The grid barrier alone: rounds barriers over grid blocks of one
// cooperative launch, each expecting extra arrivals more than the grid
// makes (extra > 0: the first wait runs out and sets kFlagTimeout in *flags).
cudaError_t launch_barrier_probe(int grid, unsigned extra, int rounds, unsigned long long limit_ns,
                                 unsigned* count, unsigned* flags, cudaStream_t s);
void launch_ingest(int32_t N, int32_t j0, int32_t j1, int64_t e_base, const int64_t* row_ptr,
                   const int32_t* col_in, const void* w_in, const void* w2_in, int32_t w_dtype,
                   const uint8_t* delay_in, uint16_t* rec, int32_t dmax, int32_t seg_stride,
                   void* seg, int32_t seg_kind, int32_t* indeg, unsigned* wmax_bits, unsigned* err,
                   cudaStream_t s);
void launch_max_reduce(const int32_t* a, int64_t n, unsigned* out, cudaStream_t s);
// adds to *out the out-degrees of the spikes handed on at steps g - 1 ..
// g - 1 + bin_lead, which no delivery has counted yet
void launch_pending_events(const EngineDev& e, unsigned long long g, unsigned long long* out,
                           cudaStream_t s);

enum : unsigned {
  kErrTarget = 1u,
  kErrDelayRange = 2u,
  kErrDelayOrder = 4u,
  kErrWeight = 8u,
  kErrRounded = 16u,
};

}  // namespace dbn

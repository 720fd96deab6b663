// Hot-path kernels for sm_103a.
//
//   k_update   one Euler step of every neuron (Methods, capacitance-voltage
//              equation and Eq. 2; Supplementary Sec. 3, Eqs. 3 and 5 with
//              the refractory reset), the Poisson background drawn from
//              Philox4x64-10, spike compaction into the spike ring,
//              and region spike counts; k_update<true> also integrates the
//              background OU current (Eq. 1) and applies the per-neuron
//              injected-current factors; k_update<., true> reads four
//              accumulator channels (two weights per edge) instead of the
//              two classes.
//   k_close / the head of k_deliver: the per-bin Balloon-Windkessel step
//              (Extended Data Table 4) and the BOLD sample, one region per
//              thread.
//   k_deliver  push delivery (Supplementary Algorithm 2) at arrival time: for
//              every spike of step n - d (d = 1..D-1, from the spike ring)
//              the edges of its row with delay exactly d -- one contiguous
//              segment, read from the delay-major segment ring that the
//              leading blocks fill for the previous step's spikes (or from
//              the graph's segment table) -- are added to this step's
//              fixed-point accumulators, the warp's segments laid end to end
//              so that consecutive lanes read consecutive edge records;
//              k_deliver<true> adds an edge's two weights to the channel pair
//              of the source's class with one 64-bit atomic.
//
// Both kernels find their iteration through a StepRef (a base word in device
// memory plus an offset), so a captured CUDA graph of (deliver, update) pairs
// is valid for any step.  The bin that ends with an iteration is closed (BW
// step, BOLD sample) by the next k_deliver, or by k_close at the end of a
// step call.
//
// The FP32 neuron arithmetic is written with explicit round-to-nearest
// intrinsics in a fixed order so that no operation is fused or reordered; the
// library is also built with -fmad=false.
#include <cuda_runtime.h>

#include "engine.h"

namespace dbn {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// (philox4x64_10 is in engine.h: the host draws with it too)

__device__ __forceinline__ int find_region(const int32_t* __restrict__ ro, int R, int32_t li) {
  int lo = 0, hi = R - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(ro + mid) <= li) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Edge records stream through the delivery once (a spike's row is read in a
// few short segments, one per delay, spread over up to D steps), while the
// accumulators of the step are its working set: the record loads carry an
// L2 evict-first policy and the accumulator reductions an evict-last one
// (PTX createpolicy / .L2::cache_hint).
#ifndef DBNET_L2_HINTS
#define DBNET_L2_HINTS 1
#endif
// 32-edge chunks of a warp's walk whose record loads are issued before the
// first of their atomics (memory-level parallelism of the walk).
#ifndef DBNET_WALK_CHUNKS
#define DBNET_WALK_CHUNKS 4
#endif
constexpr int kWalkU = DBNET_WALK_CHUNKS;
constexpr int kSegGroup = 32;  // spikes per transposition group of the segment-ring copy
constexpr int kMaxPhases = 8;  // rank phases of the arrival items (see k_deliver)

__device__ __forceinline__ unsigned long long l2_policy_first() {
  unsigned long long p = 0;
#if DBNET_L2_HINTS
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
#endif
  return p;
}
__device__ __forceinline__ unsigned long long l2_policy_last() {
  unsigned long long p = 0;
#if DBNET_L2_HINTS
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
#endif
  return p;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const uint32_t* a, unsigned long long pol) {
#if DBNET_L2_HINTS
  uint32_t v;
  asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
#else
  (void)pol;
  return __ldg(a);
#endif
}
__device__ __forceinline__ uint2 ld_stream_u64(const uint2* a, unsigned long long pol) {
#if DBNET_L2_HINTS
  uint2 v;
  asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(a), "l"(pol));
  return v;
#else
  (void)pol;
  return __ldg(a);
#endif
}
__device__ __forceinline__ void red_add_s32(int* a, int v, unsigned long long pol) {
#if DBNET_L2_HINTS
  asm volatile("red.global.add.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol));
#else
  (void)pol;
  atomicAdd(a, v);
#endif
}
__device__ __forceinline__ void red_add_u64(unsigned long long* a, unsigned long long v,
                                            unsigned long long pol) {
#if DBNET_L2_HINTS
  asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(a), "l"(v), "l"(pol));
#else
  (void)pol;
  atomicAdd(a, v);
#endif
}

// Forward-Euler step of the hemodynamic model for one region (FP64).
__device__ double bw_euler(double* x, double z, const InstDesc& d) {
  const double s = x[0], f = x[1], v = x[2], q = x[3];
  const double fout = pow(v, 1.0 / d.alpha);
  const double E = 1.0 - pow(1.0 - d.rho, 1.0 / f);
  const double ds = z - d.kappa * s - d.gamma * (f - 1.0);
  const double dv = (f - fout) / d.tau;
  const double dq = (f * E / d.rho - fout * q / v) / d.tau;
  const double h = d.h_bw;
  const double s2 = s + h * ds, f2 = f + h * s, v2 = v + h * dv, q2 = q + h * dq;
  x[0] = s2;
  x[1] = f2;
  x[2] = v2;
  x[3] = q2;
  const double k1 = 7.0 * d.rho, k2 = 2.0, k3 = 2.0 * d.rho - 0.2;
  return d.V0 * (k1 * (1.0 - q2) + k2 * (1.0 - q2 / v2) + k3 * (1.0 - v2));
}

__global__ void __launch_bounds__(kUpdThreads) k_init_state(EngineDev e, int inst, int first_tile) {
  const InstDesc& d = e.insts[inst];
  const int64_t gi0 = (int64_t)(first_tile + blockIdx.x) * kTile + threadIdx.x * 4;
  const int32_t li0 = (int32_t)(gi0 - d.base);
  float v4[4] = {0.f, 0.f, 0.f, 0.f};
  float b4[4] = {0.f, 0.f, 0.f, 0.f};  // background OU current starts at its mean
  unsigned long long c[4] = {0ull, (unsigned long long)(li0 >> 2), 1ull, 0ull};
  philox4x64_10(c, d.seed, d.net_id);
  int r = li0 < d.N ? find_region(d.region_offsets, d.R, li0) : 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int32_t li = li0 + k;
    if (li < d.N) {
      while (li >= d.rc[r].end) ++r;
      const RegionConst& p = d.rc[r];
      const float u = __fmul_rn(__ull2float_rn(c[k] >> 40), 5.9604644775390625e-08f);  // 2^-24
      const float span = __fsub_rn(p.Vth, p.Vreset);
      v4[k] = __fadd_rn(p.Vreset, __fmul_rn(span, u));
      if (p.ext & kExtOU) b4[k] = p.ou_mu;
    }
  }
  *reinterpret_cast<float4*>(e.V + gi0) = make_float4(v4[0], v4[1], v4[2], v4[3]);
  if (e.Ibg) *reinterpret_cast<float4*>(e.Ibg + gi0) = make_float4(b4[0], b4[1], b4[2], b4[3]);
#pragma unroll
  for (int u = 0; u < 4; ++u)
    *reinterpret_cast<float4*>(e.J + u * e.stride + gi0) = make_float4(0.f, 0.f, 0.f, 0.f);
  *reinterpret_cast<uint32_t*>(e.ref + gi0) = 0u;
  // accumulators: int2 per neuron, or int4 (acc[2i], acc[2i + 1]) with four
  // channels, in every slot of the ring
  const int words = e.four ? 4 : 2;
  for (int a = 0; a < e.acc_slots; ++a) {
    int2* slot = e.acc + (size_t)a * (size_t)e.stride * (e.four ? 2 : 1);
    for (int k = 0; k < words; ++k)
      *reinterpret_cast<int4*>(slot + (e.four ? 2 : 1) * gi0 + 2 * k) = make_int4(0, 0, 0, 0);
  }
}

__device__ __forceinline__ unsigned long long step_of(const StepRef& sr) {
  return (sr.base ? *reinterpret_cast<const volatile unsigned long long*>(sr.base) : 0ull) + sr.off;
}

// Close the bin that ended with iteration g - 1 for region gr, once: the
// Balloon-Windkessel step with that bin's activity, and the BOLD sample when
// the bin ends a TR.
__device__ void close_region(const EngineDev& e, int gr, unsigned long long g) {
  const int k = e.region_inst[gr];
  if (k < 0 || !e.dyn[k].active) return;  // unused region slot, or retired
  const InstDesc& dk = e.insts[k];
  if (g <= dk.g0) return;
  const long long nk = (long long)(g - 1ull - dk.g0);  // step just completed
  if (nk >= dk.n_end) return;                          // past the instance's last step
  if ((nk + 1) % dk.spb != 0) return;
  if (e.closed[gr] >= (long long)g) return;
  const int r = gr - dk.rbase;
  const double nr = (double)(dk.rc[r].end - dk.rc[r].start);
  const double z = dk.z_scale * (double)e.cnt[gr] / nr;
  e.cnt[gr] = 0;
  const double y = bw_euler(e.bw + 4 * gr, z, dk);
  e.ylast[gr] = y;
  const long long b = (nk + 1) / dk.spb;  // bins completed
  if (b % dk.bins_per_tr == 0) {
    const long long sidx = b / dk.bins_per_tr - 1;
    if (sidx < dk.bold_cap) dk.bold[sidx * dk.R + r] = y;
  }
  e.closed[gr] = (long long)g;
}

__global__ void k_close(EngineDev e, unsigned long long g) {
  for (int gr = blockIdx.x * blockDim.x + threadIdx.x; gr < e.total_R; gr += gridDim.x * blockDim.x)
    close_region(e, gr, g);
}

__global__ void k_set_base(unsigned long long* base, unsigned long long g) { *base = g; }

// Standard normal from one Philox word (Box-Muller): u1 = (high 32 bits + 1)
// 2^-32 in (0, 1], u2 = low 32 bits 2^-32, sqrt(-2 ln u1) cos(2 pi u2) in FP32.
__device__ __forceinline__ float normal_from_word(unsigned long long w) {
  const float u1 = __double2float_rn(((double)(uint32_t)(w >> 32) + 1.0) * 2.3283064365386963e-10);
  const float u2 = __double2float_rn((double)(uint32_t)w * 2.3283064365386963e-10);
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

// EXT: also the kExt* terms of the instances that have them: the background
// OU current and the per-neuron injected-current factor.  FOUR: the
// accumulators hold four channels per neuron (two weights per edge); the
// background drive adds to both AMPA and NMDA.
//
// One tile of the iteration sr names; the block's threads call it together.
template <bool EXT, bool FOUR>
__device__ __forceinline__ void update_tile(const EngineDev& e, const StepRef& sr, int tile) {
  __shared__ RegionConst s_rc[kTileRegions];
  __shared__ uint32_t s_wtot[kUpdThreads / 32];
  __shared__ uint32_t s_hbase;
  __shared__ unsigned long long s_rbase;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // state loads first: they depend only on the tile, and the arrays cover
  // every padded tile
  const int64_t gi0 = (int64_t)tile * kTile + threadIdx.x * 4;
  // (state is streamed once per step: evict-first, so that the delivery's
  // working set keeps the L2)
  const float4 V4 = __ldcs(reinterpret_cast<const float4*>(e.V + gi0));
  float4 J4[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) J4[u] = __ldcs(reinterpret_cast<const float4*>(e.J + u * e.stride + gi0));
  const uchar4 rf = __ldcs(reinterpret_cast<const uchar4*>(e.ref + gi0));
  float4 B4 = make_float4(0.f, 0.f, 0.f, 0.f), F4 = make_float4(1.f, 1.f, 1.f, 1.f);
  if (EXT) {
    B4 = __ldcs(reinterpret_cast<const float4*>(e.Ibg + gi0));
    F4 = __ldg(reinterpret_cast<const float4*>(e.fext + gi0));
  }
  // this step's arrivals, per channel (AMPA, NMDA, GABA_A, GABA_B) of the
  // thread's four neurons, from the accumulator slot of this iteration
  const unsigned long long g = step_of(sr);
  int2* const accs = e.acc + (e.acc_slots > 1 ? (size_t)(g % (unsigned long long)e.acc_slots) : 0) *
                                 (size_t)e.stride * (FOUR ? 2 : 1);
  int4 A[4];
  if (FOUR) {
#pragma unroll
    for (int k = 0; k < 4; ++k) A[k] = *reinterpret_cast<const int4*>(accs + 2 * gi0 + 2 * k);
  } else {
    const int4 a01 = *reinterpret_cast<const int4*>(accs + gi0);
    const int4 a23 = *reinterpret_cast<const int4*>(accs + gi0 + 2);
    A[0] = make_int4(a01.x, a01.x, a01.y, a01.y);
    A[1] = make_int4(a01.z, a01.z, a01.w, a01.w);
    A[2] = make_int4(a23.x, a23.x, a23.y, a23.y);
    A[3] = make_int4(a23.z, a23.z, a23.w, a23.w);
  }

  const int4 ti = e.tile_info[tile];  // instance, first region, regions touched
  if (sr.next && threadIdx.x == 0) *sr.next = g + 1ull;
  if (ti.x < 0) return;  // unused tile
  const int inst = ti.x, r0 = ti.y, nr = ti.z;
  const InstDesc& d = e.insts[inst];
  const long long n = (long long)(g - d.g0);
  const bool active = e.dyn[inst].active != 0 && n < d.n_end;
  if (nr <= kTileRegions) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(d.rc + r0);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_rc);
    const int words = nr * (int)(sizeof(RegionConst) / 4);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  const RegionConst* rcp = nr <= kTileRegions ? s_rc : d.rc + r0;

  const int32_t li0 = (int32_t)(gi0 - d.base);
  unsigned spk = 0;       // bit k: neuron li0 + k spiked
  unsigned cls_bits = 0;  // bit k: that neuron is inhibitory
  int reg[4] = {0, 0, 0, 0};

  if (active && li0 < d.N) {
#pragma unroll
    for (int k = 0; k < (FOUR ? 4 : 2); ++k)
      *reinterpret_cast<int4*>(accs + (FOUR ? 2 : 1) * gi0 + 2 * k) = make_int4(0, 0, 0, 0);
    unsigned long long x[4] = {(unsigned long long)n, (unsigned long long)(li0 >> 2), 0ull, 0ull};
    philox4x64_10(x, d.seed, d.net_id);
    float ib[4] = {B4.x, B4.y, B4.z, B4.w};
    const float fe[4] = {F4.x, F4.y, F4.z, F4.w};
    unsigned long long xo[4] = {0ull, 0ull, 0ull, 0ull};
    if (EXT && (d.ext & kExtOU)) {  // the OU noise: stream 4
      xo[0] = (unsigned long long)n;
      xo[1] = (unsigned long long)(li0 >> 2);
      xo[2] = 4ull;
      philox4x64_10(xo, d.seed, d.net_id);
    }

    float v[4] = {V4.x, V4.y, V4.z, V4.w};
    float j[4][4] = {{J4[0].x, J4[0].y, J4[0].z, J4[0].w},
                     {J4[1].x, J4[1].y, J4[1].z, J4[1].w},
                     {J4[2].x, J4[2].y, J4[2].z, J4[2].w},
                     {J4[3].x, J4[3].y, J4[3].z, J4[3].w}};
    int rr[4] = {rf.x, rf.y, rf.z, rf.w};
    int r = 0;  // relative to r0
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int32_t li = li0 + k;
      if (li >= d.N) break;
      while (li >= rcp[r].end) ++r;
      reg[k] = r0 + r;
      const RegionConst& p = rcp[r];
      const float4 G = *reinterpret_cast<const float4*>(p.g);
      const float4 VU = *reinterpret_cast<const float4*>(p.Vu);
      const float4 DE = *reinterpret_cast<const float4*>(p.dec);
      const float4 M = *reinterpret_cast<const float4*>(&p.dtC);     // dtC gL VL Vth
      const float4 Q = *reinterpret_cast<const float4*>(&p.Vreset);  // Vreset Iext n_ref q_ext
      const int4 W = *reinterpret_cast<const int4*>(&p.n_thr);       // n_thr exc_end start end
      // background: Poisson count by integer inversion of 32 Philox bits
      // (the thresholds are non-decreasing: count them up to the first miss)
      const uint32_t uu = (uint32_t)(x[k] >> 32);
      int c = 0;
      while (c < W.x && uu >= p.thr[c]) ++c;
      const int dq = c * __float_as_int(Q.w);
      const int a0 = A[k].x + dq, a1 = A[k].y + dq;  // the drive feeds AMPA and NMDA
      // membrane with the old V and traces
      const float vk = v[k];
      const float gu[4] = {G.x, G.y, G.z, G.w}, vu[4] = {VU.x, VU.y, VU.z, VU.w};
      float Isyn = 0.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float gj = __fmul_rn(gu[u], j[u][k]);
        const float dv = __fsub_rn(vu[u], vk);
        Isyn = __fadd_rn(Isyn, __fmul_rn(gj, dv));
      }
      const float leak = __fmul_rn(M.y, __fsub_rn(vk, M.z));
      float I = __fsub_rn(Isyn, leak);
      float4 OUc = make_float4(0.f, 0.f, 0.f, 0.f);  // mu, dt/tau, sigma sqrt(2 dt/tau), bits
      if (EXT && d.ext) OUc = *reinterpret_cast<const float4*>(&p.ou_mu);
      const int xb = __float_as_int(OUc.w);
      // injected current, scaled by the neuron's factor where heterogeneous
      const float ie = (EXT && (xb & kExtHet)) ? __fmul_rn(Q.y, fe[k]) : Q.y;
      I = __fadd_rn(I, ie);
      if (EXT && (xb & kExtOU)) I = __fadd_rn(I, ib[k]);  // I_bg before this step
      const float vn = __fadd_rn(vk, __fmul_rn(I, M.x));
      if (EXT && (xb & kExtOU)) {  // Eq. 1, Euler-Maruyama
        const float xi = normal_from_word(xo[k]);
        const float t1 = __fmul_rn(__fsub_rn(OUc.x, ib[k]), OUc.y);
        ib[k] = __fadd_rn(ib[k], t1);
        ib[k] = __fadd_rn(ib[k], __fmul_rn(OUc.z, xi));
      }
      // traces: decay, then this step's arrivals
      const float x0 = __fmul_rn(__int2float_rn(a0), d.inv_two_S);
      const float x1 = FOUR ? __fmul_rn(__int2float_rn(a1), d.inv_two_S) : x0;
      const float x2 = __fmul_rn(__int2float_rn(A[k].z), d.inv_two_S);
      const float x3 = FOUR ? __fmul_rn(__int2float_rn(A[k].w), d.inv_two_S) : x2;
      j[0][k] = __fadd_rn(__fmul_rn(DE.x, j[0][k]), x0);
      j[1][k] = __fadd_rn(__fmul_rn(DE.y, j[1][k]), x1);
      j[2][k] = __fadd_rn(__fmul_rn(DE.z, j[2][k]), x2);
      j[3][k] = __fadd_rn(__fmul_rn(DE.w, j[3][k]), x3);
      // refractory clamp, threshold, reset
      if (rr[k] > 0) {
        v[k] = Q.x;
        rr[k] -= 1;
      } else if (vn >= M.w) {
        v[k] = Q.x;
        rr[k] = __float_as_int(Q.z);
        spk |= 1u << k;
        if (li >= W.y) cls_bits |= 1u << k;
      } else {
        v[k] = vn;
      }
    }
    __stcs(reinterpret_cast<float4*>(e.V + gi0), make_float4(v[0], v[1], v[2], v[3]));
#pragma unroll
    for (int u = 0; u < 4; ++u)
      __stcs(reinterpret_cast<float4*>(e.J + u * e.stride + gi0),
             make_float4(j[u][0], j[u][1], j[u][2], j[u][3]));
    __stcs(reinterpret_cast<uchar4*>(e.ref + gi0),
           make_uchar4((unsigned char)rr[0], (unsigned char)rr[1], (unsigned char)rr[2],
                       (unsigned char)rr[3]));
    if (EXT && (d.ext & kExtOU))
      __stcs(reinterpret_cast<float4*>(e.Ibg + gi0), make_float4(ib[0], ib[1], ib[2], ib[3]));
  }

  // ---- spikes: one ring append, spike and raster count per block ---------
  if (!__syncthreads_or(spk != 0)) return;
  const int nsp = __popc(spk);
  int ps = nsp;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, ps, o);
    if (lane >= o) ps += t;
  }
  if (lane == 31) s_wtot[warp] = (uint32_t)ps;
  __syncthreads();
  // the ring slot of the step at which these spikes are handed on: this
  // step, or with spike binning the last step of its bin
  const unsigned long long rel =
      d.bin_sp ? d.g0 + (unsigned long long)((n / d.spb + 1) * d.spb - 1) : g;
  const int slot = (int)(rel % (unsigned long long)e.D);
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int w = 0; w < kUpdThreads / 32; ++w) {
      const uint32_t c = s_wtot[w];
      s_wtot[w] = tot;  // exclusive prefix
      tot += c;
    }
    s_hbase = atomicAdd(e.hcount + slot, tot);
    atomicAdd(&e.dyn[inst].spikes, (unsigned long long)tot);
    s_rbase = d.raster_cap > 0 ? atomicAdd(&e.dyn[inst].raster_count, (unsigned long long)tot) : 0ull;
  }
  __syncthreads();
  if (spk) {
    uint64_t pos = (uint64_t)s_hbase + s_wtot[warp] + (uint32_t)(ps - nsp);
    unsigned long long rpos = s_rbase + s_wtot[warp] + (unsigned long long)(ps - nsp);
    uint32_t* hslot = e.hist + (size_t)slot * (size_t)e.hist_cap;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!(spk & (1u << k))) continue;
      if (pos < (uint64_t)e.hist_cap)
        hslot[pos] = (uint32_t)(gi0 + k) | (((cls_bits >> k) & 1u) << 31);
      else
        atomicOr(e.flags, kFlagHistOverflow);
      ++pos;
      atomicAdd(&e.cnt[d.rbase + reg[k]], 1);
      if (d.raster_cap > 0) {
        if (rpos < (unsigned long long)d.raster_cap) {
          d.raster_step[rpos] = (int32_t)n;
          d.raster_id[rpos] = li0 + k;
        }
        ++rpos;
      }
    }
  }
}

template <bool EXT, bool FOUR>
__global__ void __launch_bounds__(kUpdThreads, 4) k_update(EngineDev e, StepRef sr) {
  update_tile<EXT, FOUR>(e, sr, blockIdx.x);
}

__device__ __forceinline__ uint32_t edge_delay(const uint32_t* col, const uint8_t* dl, int shift,
                                               int64_t e) {
  return dl ? (uint32_t)__ldg(dl + e) : (__ldg(col + e) >> shift);
}

// first edge in [lo, hi) whose delay is >= d (rows are sorted by delay)
__device__ int64_t first_delay_at_least(const uint32_t* col, const uint8_t* dl, int shift,
                                        int64_t lo, int64_t hi, uint32_t d) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (edge_delay(col, dl, shift, mid) < d) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Stage one of resolving an item (spike k of the ring slot of step g - d,
// delay d, due now; or, in the emission range, spike k of step g - 1 and one
// of its long delays d): everything that needs no other load -- the ring
// entry and, from the delay-major segment ring, the row start and the two
// segment counts -- and the accumulator slot its edges go to.
struct ItemLoads {
  uint32_t ent, d, slot, k, aslot;
  int64_t r0;
  uint32_t a, b;
  bool ring;
};

// FOUR: the engine keeps four accumulator channels per neuron; an edge adds
// its two weights (the one weight twice for one-weight records) to the
// channel pair of the source's class with one 64-bit atomic.  Every channel
// sum stays below 2^31 (the fixed-point scale is chosen so), so the low word
// never carries into the high one.  SINGLE: the engine holds one instance
// (a network, or the allocation-free run), so every spike's descriptor is
// the first.
// part: kPartAll does the whole delivery of iteration g.  The pipelined
// schedule splits it: kPartLong, the arrival items of delays >= 2, which
// read only spikes of steps <= g - 2 and so run beside the update of
// iteration g - 1; then kPartShort after that update: the bin close, the
// ring bookkeeping, the segment-ring copy of step g - 1's spikes, the
// delay-1 items and the emission items.
// Loads of the spike and segment rings: through the read-only path when
// the rings are written only by earlier launches; from the L2 (coherent,
// never a stale L1 line) in the persistent stepper, whose own blocks wrote
// them earlier in the launch.
template <bool PERSIST, typename T>
__device__ __forceinline__ T ld_ring(const T* p) {
  if (PERSIST) return __ldcg(p);
  return __ldg(p);
}

// The delivery of the iteration sr names, as block bid of nblk; the block's
// threads call it together.
template <bool FOUR, bool SINGLE, bool PERSIST>
__device__ __forceinline__ void deliver_body(const EngineDev& e, const StepRef& sr, int part, int bid,
                                             int nblk) {
  // arrival items of phase q and delay bucket i start at s_phase[q] +
  // s_pre[q][i]; bucket i holds ranks [q c/Q, (q+1) c/Q) of the c spikes
  // handed on at g - i - 1
  __shared__ unsigned long long s_pre[kMaxPhases][256];
  __shared__ unsigned long long s_wsum[kMaxPhases][kDelThreads / 32];
  __shared__ unsigned long long s_phase[kMaxPhases + 1];
  __shared__ uint32_t s_cnt[256];
  __shared__ __align__(16) uint16_t s_tab[256 * kSegGroup];  // [delay][spike] of a copy group
  __shared__ const uint4* s_row[kSegGroup];
  __shared__ int32_t s_nq[kSegGroup];
  __shared__ long long s_r0[kSegGroup];
  const unsigned long long g = step_of(sr);
  const int D = e.D;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gtid = bid * blockDim.x + threadIdx.x;
  // close the bin that ended with the previous iteration, one region per thread
  const bool do_short = part != kPartLong, do_long = part != kPartShort;
  if (do_short)
    for (int gr = gtid; gr < e.total_R; gr += nblk * blockDim.x) close_region(e, gr, g);
  // the slot that the updates from this iteration on fill (a bin later with
  // spike binning) was last read by the previous iteration; the slot handed
  // on at g - 1 gets its long delays now, at emission, when d_emit allows
  const unsigned long long s1 = (g + (unsigned long long)D - 1ull) % (unsigned long long)D;
  if (gtid == 0 && do_short) {
    e.hcount[(g + (unsigned long long)e.bin_lead) % (unsigned long long)D] = 0u;
    if (e.slot_emit) e.slot_emit[s1] = (uint16_t)e.d_emit;
  }
  // The leading nA blocks copy the row start and segment counts of the
  // previous step's spikes into the delay-major ring and take no items; nA
  // follows that step's spike count, the same in every block.
  unsigned long long c1 = 0;
  int nA = 0;
  // delay-major planes the later arrival items read: delays below d_emit
  const int planes = e.dcap < e.d_emit - 1 ? e.dcap : e.d_emit - 1;
  if (e.seg_cap > 0 && g >= 1ull && planes > 1 && do_short) {
    c1 = e.hcount[s1];
    if (c1 > (unsigned long long)e.hist_cap) c1 = (unsigned long long)e.hist_cap;
    if (c1 > (unsigned long long)e.seg_cap) c1 = (unsigned long long)e.seg_cap;
    const unsigned long long want = (c1 + kSegGroup - 1) / kSegGroup;
    // at most a 32nd of the grid: the copy overlaps the item blocks' work
    const int most = nblk >= 64 ? nblk / 32 : 1;  // the host launches >= 2 blocks
    nA = want < (unsigned long long)most ? (int)want : most;
  }
  if (bid < nA) {
    // Groups of 32 spikes: their segment-table rows are loaded at once (one
    // 16-byte vector of 8 delays per task, consecutive lanes on consecutive
    // spikes), transposed in shared memory to [delay][spike], and stored
    // plane by plane, 64 contiguous bytes per delay.
    const size_t cap = (size_t)e.seg_cap;
    const int dcap = e.dcap;
    const int nq_all = (planes + 7) >> 3;
    for (unsigned long long k0 = (unsigned long long)bid * kSegGroup; k0 < c1;
         k0 += (unsigned long long)nA * kSegGroup) {
      if (threadIdx.x < kSegGroup) {
        const unsigned long long k = k0 + threadIdx.x;
        const uint4* row = nullptr;
        int nq = 0;
        long long r0 = 0;
        if (k < c1) {
          const uint32_t ent = ld_ring<PERSIST>(e.hist + s1 * (unsigned long long)e.hist_cap + k);
          const int64_t gidx = (int64_t)(ent & 0x7FFFFFFFu);
          const int inst = SINGLE ? 0 : e.tile_info[gidx / kTile].x;
          if (inst >= 0) {
            const InstDesc& dd = e.insts[inst];
            if (dd.seg_kind == kSeg16) {
              const int64_t j = gidx - dd.base;
              r0 = __ldg(dd.row_ptr + j);
              row = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(dd.seg) +
                                                   j * dd.seg_stride);
              nq = (dd.dmax + 7) >> 3;
            }
          }
        }
        s_row[threadIdx.x] = row;
        s_nq[threadIdx.x] = nq;
        s_r0[threadIdx.x] = r0;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < kSegGroup * nq_all; t += kDelThreads) {
        const int ks = t & (kSegGroup - 1), q = t / kSegGroup;
        const uint4 v = q < s_nq[ks] ? __ldg(s_row[ks] + q) : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
          s_tab[(8 * q + i) * kSegGroup + ks] = (uint16_t)(wd[i >> 1] >> ((i & 1) * 16));
      }
      __syncthreads();
      // k0 + 31 < seg_cap (a multiple of 32): whole groups stay in the ring
      for (int t = threadIdx.x; t < planes * (kSegGroup / 2); t += kDelThreads) {
        const int dl = t / (kSegGroup / 2), w = t % (kSegGroup / 2);
        const uint32_t pair = *reinterpret_cast<const uint32_t*>(&s_tab[dl * kSegGroup + 2 * w]);
        uint32_t* H = reinterpret_cast<uint32_t*>(e.hseg + (s1 * (size_t)dcap + dl) * cap + k0);
        H[w] = pair;
      }
      if (threadIdx.x < kSegGroup) e.hr0[s1 * cap + k0 + threadIdx.x] = s_r0[threadIdx.x];
      __syncthreads();
    }
    return;
  }
  const int bB = bid - nA, nB = nblk - nA;  // item blocks

  // spikes handed on at step g - d for d = threadIdx.x + 1, and their
  // exclusive prefix (delays up to D - 1 - bin_lead: the later slots hold
  // bins still filling)
  const int dlim = D - 1 - e.bin_lead;
  unsigned long long c = 0;
  const int dme = threadIdx.x + 1;
  if (dme <= dlim && g >= (unsigned long long)dme && (dme == 1 ? do_short : do_long)) {
    const unsigned long long sl = (g - dme) % (unsigned long long)D;
    // delays at or above the threshold in force when that slot was handed
    // on went out at emission
    const int thr = dme == 1 ? e.d_emit : (e.slot_emit ? (int)e.slot_emit[sl] : D + 1);
    if (dme < thr) {
      const unsigned long long h = e.hcount[sl];
      c = h < (unsigned long long)e.hist_cap ? h : (unsigned long long)e.hist_cap;
    }
  }
  // Phases: the update appends each step's spikes roughly in tile order, so
  // a spike's rank in its slot follows its region.  Taking the items rank
  // phase by rank phase (phase q: ranks [q c/Q, (q+1) c/Q) of every delay's
  // slot) keeps the warps in flight on a narrow band of regions, so the
  // within-region edges (most of them) add into a slice of the accumulators
  // that stays in the L2 even when all of them do not fit (Q = 1 when they
  // do).
  const int Q = e.phases;
  s_cnt[threadIdx.x] = (uint32_t)c;
  unsigned long long incl[kMaxPhases], own[kMaxPhases];
#pragma unroll
  for (int q = 0; q < kMaxPhases; ++q) {
    own[q] = q < Q ? (q + 1ull) * c / (unsigned long long)Q - q * c / (unsigned long long)Q : 0ull;
    incl[q] = own[q];
    if (q < Q) {  // block-uniform
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(kFull, incl[q], o);
        if (lane >= o) incl[q] += t;
      }
    }
    if (lane == 31) s_wsum[q][warp] = incl[q];
  }
  __syncthreads();
  if (threadIdx.x < kMaxPhases) {  // warp offsets within each phase
    unsigned long long acc = 0;
    for (int w = 0; w < kDelThreads / 32; ++w) {
      const unsigned long long t = s_wsum[threadIdx.x][w];
      s_wsum[threadIdx.x][w] = acc;
      acc += t;
    }
    s_phase[threadIdx.x + 1] = acc;  // the phase's total, summed below
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_phase[0] = 0ull;
    for (int q = 0; q < kMaxPhases; ++q) s_phase[q + 1] += s_phase[q];
  }
#pragma unroll
  for (int q = 0; q < kMaxPhases; ++q) s_pre[q][threadIdx.x] = s_wsum[q][warp] + incl[q] - own[q];
  __syncthreads();
  const int nd = dlim < kDelThreads ? dlim : kDelThreads;  // delay buckets d = 1..nd
  // the emission range: every spike handed on at g - 1 times its delays
  // d_emit..dlim, spike-major so that consecutive lanes take consecutive
  // delays of one row (its segments lie end to end)
  const unsigned long long W_arr = s_phase[Q];
  const int ne = e.d_emit <= dlim ? dlim - e.d_emit + 1 : 0;
  unsigned long long c1e = 0;
  if (ne > 0 && g >= 1ull && do_short) {
    c1e = e.hcount[s1];
    if (c1e > (unsigned long long)e.hist_cap) c1e = (unsigned long long)e.hist_cap;
  }
  const unsigned long long W = W_arr + c1e * (unsigned long long)ne;
  const unsigned long long acc_elems = (unsigned long long)e.stride * (FOUR ? 2 : 1);
  const uint32_t aslot_now = e.acc_slots > 1 ? (uint32_t)(g % (unsigned long long)e.acc_slots) : 0u;
  __syncthreads();

  const unsigned long long pol_rec = l2_policy_first(), pol_acc = l2_policy_last();
  const size_t cap = (size_t)e.seg_cap;
  // stage one: bucket (delay) by binary search over the prefix, then the
  // loads that need nothing else
  auto stage_one = [&](unsigned long long t, ItemLoads& p) {
    p.d = 0u;
    p.ring = false;
    if (t >= W) return;
    if (t >= W_arr) {  // emission: spike k of step g - 1, delay d, into slot g - 1 + d
      const unsigned long long te = t - W_arr;
      p.k = (uint32_t)(te / (unsigned long long)ne);
      p.d = (uint32_t)e.d_emit + (uint32_t)(te % (unsigned long long)ne);
      p.slot = (uint32_t)s1;
      p.aslot = (uint32_t)((g - 1ull + p.d) % (unsigned long long)e.acc_slots);
      p.ent = ld_ring<PERSIST>(e.hist + (size_t)p.slot * (size_t)e.hist_cap + p.k);
      return;
    }
    p.aslot = aslot_now;
    int q = 0;  // the phase: the largest q < Q with s_phase[q] <= t
    for (int step = kMaxPhases / 2; step > 0; step >>= 1)
      if (q + step < Q && s_phase[q + step] <= t) q += step;
    const unsigned long long tq = t - s_phase[q];
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_pre[q][mid] <= tq) lo = mid; else hi = mid - 1;
    }
    p.d = (uint32_t)lo + 1u;
    p.k = (uint32_t)((unsigned long long)q * s_cnt[lo] / (unsigned long long)Q + (tq - s_pre[q][lo]));
    p.slot = (uint32_t)((g - p.d) % (unsigned long long)D);
    p.ent = ld_ring<PERSIST>(e.hist + (size_t)p.slot * (size_t)e.hist_cap + p.k);
    if (p.d >= 2u && p.k < cap) {  // from the delay-major ring (coalesced across lanes)
      p.ring = true;
      p.r0 = ld_ring<PERSIST>(e.hr0 + p.slot * cap + p.k);
      const uint16_t* H = e.hseg + ((size_t)p.slot * (size_t)e.dcap) * cap + p.k;
      p.a = ld_ring<PERSIST>(H + (size_t)(p.d - 2u) * cap);
      p.b = ld_ring<PERSIST>(H + (size_t)(p.d - 1u) * cap);
    }
  };
  // stage two: the item's edge segment [e0, e0 + nseg) from the stage-one
  // loads, or by the graph's own tables when the ring does not hold it
  // The synaptic events of a spike (its out-degree: Supp. Alg. 2 pushes
  // every out-edge once) are counted at its delay-1 item, which every spike
  // handed on has exactly once (arrival, or emission when every delay goes
  // at emission); the spikes handed on at the last step, not yet reached by
  // a delivery, are added when the counters are read (k_pending_events).
  unsigned long long ev = 0;
  auto stage_two = [&](const ItemLoads& p, int64_t& e0, uint32_t& nseg, int& inst, uint32_t& cls) {
    e0 = 0;
    nseg = 0u;
    inst = 0;
    cls = 0u;
    if (p.d == 0u) return;
    cls = p.aslot << 1;  // the accumulator slot travels with the class bit
    const int64_t gidx = (int64_t)(p.ent & 0x7FFFFFFFu);
    cls |= p.ent >> 31;
    if (!SINGLE) {
      inst = e.tile_info[gidx / kTile].x;
      if (inst < 0) {  // never for a listed spike: tiles are reused D steps late
        inst = 0;
        return;
      }
    }
    const InstDesc& dd = e.insts[inst];
    const uint32_t d = p.d;
    const int64_t j = gidx - dd.base;
    if (d == 1u) ev += (unsigned long long)(__ldg(dd.row_ptr + j + 1) - __ldg(dd.row_ptr + j));
    if ((int32_t)d > dd.dmax) return;
    int64_t r0, a, b;
    if (dd.seg_kind == kSeg16 && p.ring) {
      r0 = p.r0;
      a = (int64_t)p.a;
      b = (int64_t)p.b;
    } else if (dd.seg_kind == kSeg16) {
      r0 = __ldg(dd.row_ptr + j);
      const uint16_t* T = static_cast<const uint16_t*>(dd.seg) + j * dd.seg_stride;
      a = d >= 2 ? (int64_t)__ldg(T + d - 2) : 0;
      b = (int64_t)__ldg(T + d - 1);
    } else if (dd.seg_kind == kSeg32) {
      r0 = __ldg(dd.row_ptr + j);
      const uint32_t* T = static_cast<const uint32_t*>(dd.seg) + j * dd.seg_stride;
      a = d >= 2 ? (int64_t)__ldg(T + d - 2) : 0;
      b = (int64_t)__ldg(T + d - 1);
    } else {
      r0 = __ldg(dd.row_ptr + j);
      const int64_t r1 = __ldg(dd.row_ptr + j + 1);
      a = first_delay_at_least(dd.col, dd.delay, dd.shift, r0, r1, d) - r0;
      b = first_delay_at_least(dd.col, dd.delay, dd.shift, r0 + a, r1, d + 1) - r0;
    }
    nseg = (uint32_t)(b - a);
    e0 = r0 + a;
  };

  const unsigned long long wstride = (unsigned long long)nB * blockDim.x;
  const unsigned long long wbase = (unsigned long long)bB * blockDim.x + warp * 32;
  ItemLoads pend;
  stage_one(wbase + lane, pend);
  for (unsigned long long b0 = wbase; b0 < W; b0 += wstride) {  // warp-uniform
    int64_t e0;
    uint32_t nseg, cls;
    int inst;
    stage_two(pend, e0, nseg, inst, cls);
    // the next batch's loads fly while this batch's edges are walked
    stage_one(b0 + wstride + lane, pend);
    // the warp's segments laid end to end; consecutive lanes take
    // consecutive edges (coalesced), the owning item found by a shuffle search
    uint32_t incl = nseg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += x;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    const uint32_t ex = incl - nseg;
    // instance (23 bits) | accumulator slot << 23 (8 bits) | class << 31
    const int icls = inst | (int)((cls >> 1) << 23) | (int)((cls & 1u) << 31);
    for (uint32_t f = 0; f < total; f += 32u * kWalkU) {  // warp-uniform
      uint32_t tg[kWalkU], wv[kWalkU];
      int ic[kWalkU];
      bool ok[kWalkU];
#pragma unroll
      for (int u = 0; u < kWalkU; ++u) {
        ok[u] = false;
        if (f + 32u * u < total) {  // warp-uniform
          const uint32_t fi = f + 32u * u + lane;
          int L = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int cand = L + step < 32 ? L + step : 31;
            const uint32_t v = __shfl_sync(kFull, ex, cand);
            if (L + step < 32 && v <= fi) L = cand;
          }
          const int64_t q0 = __shfl_sync(kFull, e0, L);
          const uint32_t qx = __shfl_sync(kFull, ex, L);
          ic[u] = __shfl_sync(kFull, icls, L);
          if (fi < total) {
            const InstDesc& dd = e.insts[SINGLE ? 0 : (ic[u] & 0x7FFFFF)];
            const int64_t ei = q0 + (int64_t)(fi - qx);
            if (FOUR && dd.two_w) {  // 8-byte record: target, weight | second weight << 16
              const uint2 r4 = ld_stream_u64(reinterpret_cast<const uint2*>(dd.rec) + ei, pol_rec);
              tg[u] = r4.x;
              wv[u] = r4.y;
            } else if (dd.rec) {
              // 6-byte record at byte 6 ei: two aligned words cover it (the
              // record array carries 8 bytes of padding at its end)
              const size_t byte = 6 * (size_t)ei;
              const uint32_t* w4 = reinterpret_cast<const uint32_t*>(
                  reinterpret_cast<const unsigned char*>(dd.rec) + (byte & ~size_t(3)));
              const uint32_t w0 = ld_stream_u32(w4, pol_rec), w1 = ld_stream_u32(w4 + 1, pol_rec);
              const uint32_t sh = (uint32_t)(byte & 3u) * 8u;  // 0 or 16
              tg[u] = __funnelshift_r(w0, w1, sh);
              const uint32_t wb = (w1 >> sh) & 0xFFFFu;
              wv[u] = wb | (wb << 16);
            } else {
              tg[u] = __ldg(dd.col + ei) & dd.tmask;
              const uint32_t wb = __ldg(dd.w + ei);
              wv[u] = wb | (wb << 16);
            }
            ok[u] = true;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kWalkU; ++u) {
        if (!ok[u]) continue;
        const InstDesc& dd = e.insts[SINGLE ? 0 : (ic[u] & 0x7FFFFF)];
        const uint32_t qc = (uint32_t)ic[u] >> 31;
        int2* const accs = e.acc + (size_t)(((uint32_t)ic[u] >> 23) & 0xFFu) * acc_elems;
        const int q = __float2int_rn(__fmul_rn(__uint_as_float(wv[u] << 16), dd.two_S));
        if (FOUR) {
          const int q2 = __float2int_rn(__fmul_rn(__uint_as_float(wv[u] & 0xFFFF0000u), dd.two_S));
          unsigned long long* accp = reinterpret_cast<unsigned long long*>(accs) +
                                     2 * (size_t)(dd.base + (int64_t)tg[u]) + qc;
          red_add_u64(accp, ((unsigned long long)(uint32_t)q2 << 32) | (uint32_t)q, pol_acc);
        } else {
          int* accp = reinterpret_cast<int*>(accs + dd.base) + qc;
          red_add_s32(accp + 2 * (size_t)tg[u], q, pol_acc);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ev += __shfl_down_sync(kFull, ev, o);
  if (lane == 0 && ev) atomicAdd(e.events, ev);
}

template <bool FOUR, bool SINGLE>
__global__ void __launch_bounds__(kDelThreads, 4) k_deliver(EngineDev e, StepRef sr, int part) {
  deliver_body<FOUR, SINGLE, false>(e, sr, part, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned* a, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch.  After a block barrier (which
// orders the block's earlier writes before thread 0's), thread 0 of every
// block adds one to *count with device-scope release semantics and polls it
// with acquire loads until it reaches target (the blocks of the grid times
// the barriers passed, counting this one); the block barrier after the wait
// orders the block's later reads after the acquire.  The wait is bounded:
// after limit_ns of the global timer, or as soon as another block has given
// up (kFlagTimeout set in *flags), it gives up too, sets kFlagTimeout, and
// every thread of the block gets false.
__device__ bool grid_barrier(unsigned* count, unsigned target, unsigned long long limit_ns,
                             unsigned* flags) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_add_u32(count, 1u);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    for (unsigned spin = 0; (int)(ld_acquire_u32(count) - target) < 0; ++spin) {
      if ((spin & 15u) != 15u) continue;  // the flag and the clock every 16 polls
      if (*reinterpret_cast<volatile unsigned*>(flags) & kFlagTimeout) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > limit_ns) {
        atomicOr(flags, kFlagTimeout);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The persistent stepper: iterations g0 .. g0 + nsteps - 1 in one
// cooperative launch, each the delivery (the whole grid, as in k_deliver)
// and the update (tiles dealt round robin over the blocks), with a grid
// barrier after each.  The same device functions as the two-launch step do
// the work, so the results are identical bit for bit; a barrier that gives
// up ends the launch (kFlagTimeout stays set for the host).
template <bool EXT, bool FOUR, bool SINGLE>
__global__ void __launch_bounds__(kDelThreads, 2)
    k_persist(EngineDev e, unsigned long long g0, int nsteps, unsigned* count,
              unsigned long long limit_ns) {
  unsigned target = 0;
  for (int s = 0; s < nsteps; ++s) {
    const StepRef sr{nullptr, g0 + (unsigned long long)s, nullptr};
    deliver_body<FOUR, SINGLE, true>(e, sr, kPartAll, blockIdx.x, gridDim.x);
    target += gridDim.x;
    if (!grid_barrier(count, target, limit_ns, e.flags)) return;
    for (int t = blockIdx.x; t < e.n_tiles; t += gridDim.x) {
      __syncthreads();  // the previous tile's block-shared values are read
      update_tile<EXT, FOUR>(e, sr, t);
    }
    target += gridDim.x;
    if (!grid_barrier(count, target, limit_ns, e.flags)) return;
  }
}

// The grid barrier alone, rounds times, with extra arrivals expected per
// round that no block makes when extra > 0 (the wait then runs out).
__global__ void k_barrier_probe(unsigned* count, unsigned extra, int rounds,
                                unsigned long long limit_ns, unsigned* flags) {
  unsigned target = 0;
  for (int r = 0; r < rounds; ++r) {
    target += gridDim.x + extra;
    if (!grid_barrier(count, target, limit_ns, flags)) return;
  }
}

// BF16 bit pattern of staged weight e (float32 rounded to nearest even, or
// taken as given), with the rounding and range checks of ingest.
__device__ __forceinline__ uint16_t staged_bf16(const void* w_in, int32_t w_dtype, int64_t e,
                                                unsigned& err, unsigned& wmax) {
  uint16_t wb;
  if (w_dtype == 1) {
    wb = static_cast<const uint16_t*>(w_in)[e];
  } else {
    const float f = static_cast<const float*>(w_in)[e];
    const uint32_t u = __float_as_uint(f);
    const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);  // round to nearest even
    wb = (uint16_t)(r >> 16);
    if ((uint32_t)wb << 16 != u) err |= kErrRounded;
  }
  const uint32_t wu = (uint32_t)wb << 16;
  const float wf = __uint_as_float(wu);
  if (!(wf >= 0.0f) || isinf(wf)) err |= kErrWeight;
  else wmax = max(wmax, wu);
  return wb;
}

// Ingest rows [j0, j1) of a graph from staging arrays that hold its edges
// from e_base on: warp per source row.  Checks every edge (target range,
// delay >= 1 and non-decreasing within the row, weights finite and
// non-negative after rounding to BF16), counts in-degrees, and writes
//   rec[3e .. 3e+2] = target low 16 bits, target high 16 bits, BF16 weight
//   (with second weights w2_in: rec[4e .. 4e+3], the second weight last)
//   seg[j * seg_stride + k] = number of edges of row j with delay <= k + 1
// (the segment table must be zero on entry; entries below the row's first
// delay stay zero).
__global__ void k_ingest(int32_t N, int32_t j0, int32_t j1, int64_t e_base,
                         const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_in,
                         const void* __restrict__ w_in, const void* __restrict__ w2_in,
                         int32_t w_dtype, const uint8_t* __restrict__ delay_in,
                         uint16_t* __restrict__ rec,
                         int32_t dmax, int32_t seg_stride, void* seg, int32_t kind,
                         int32_t* indeg, unsigned* wmax_bits, unsigned* err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned my_err = 0, my_wmax = 0;
  for (int64_t j = j0 + warp; j < j1; j += nwarps) {
    const int64_t a = row_ptr[j] - e_base, b = row_ptr[j + 1] - e_base;
    for (int64_t e = a + lane; e < b; e += 32) {
      const int32_t t = col_in[e];
      const unsigned d = delay_in[e];
      if (t < 0 || t >= N) my_err |= kErrTarget;
      if (d < 1u) my_err |= kErrDelayRange;
      if (e > a && delay_in[e - 1] > d) my_err |= kErrDelayOrder;
      const uint16_t wb = staged_bf16(w_in, w_dtype, e, my_err, my_wmax);
      const uint32_t tu = (uint32_t)t;
      if (w2_in) {
        const uint16_t wb2 = staged_bf16(w2_in, w_dtype, e, my_err, my_wmax);
        reinterpret_cast<uint2*>(rec)[e_base + e] = make_uint2(tu, (uint32_t)wb | ((uint32_t)wb2 << 16));
      } else {
        uint16_t* r3 = rec + 3 * (e_base + e);
        r3[0] = (uint16_t)(tu & 0xFFFFu);
        r3[1] = (uint16_t)(tu >> 16);
        r3[2] = wb;
      }
      if (t >= 0 && t < N) atomicAdd(indeg + t, 1);
    }
    // segment counts: edge p closes the delays from its own to the next edge's
    const int64_t n = b - a;
    uint16_t* T16 = static_cast<uint16_t*>(seg) + j * seg_stride;
    uint32_t* T32 = static_cast<uint32_t*>(seg) + j * seg_stride;
    for (int64_t p = lane; p < n; p += 32) {
      const int dp = (int)delay_in[a + p];
      const int dn = p + 1 < n ? (int)delay_in[a + p + 1] : dmax + 1;
      const int k0 = dp - 1 > 0 ? dp - 1 : 0;
      const int k1 = dn - 2 < dmax - 1 ? dn - 2 : dmax - 1;  // malformed rows fail creation
      for (int k = k0; k <= k1; ++k) {
        if (kind == kSeg16) T16[k] = (uint16_t)(p + 1);
        else T32[k] = (uint32_t)(p + 1);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    my_err |= __shfl_xor_sync(kFull, my_err, o);
    my_wmax = max(my_wmax, __shfl_xor_sync(kFull, my_wmax, o));
  }
  if (lane == 0) {
    if (my_err) atomicOr(err, my_err);
    atomicMax(wmax_bits, my_wmax);
  }
}

// Out-degree sum of the spikes handed on at steps [r0, r1] (the ones no
// delivery has reached yet when the counters are read), into *out.
__global__ void k_pending_events(EngineDev e, long long r0, long long r1, unsigned long long* out) {
  unsigned long long ev = 0;
  for (long long r = r0 < 0 ? 0 : r0; r <= r1; ++r) {
    const unsigned long long slot = (unsigned long long)r % (unsigned long long)e.D;
    unsigned long long c = e.hcount[slot];
    if (c > (unsigned long long)e.hist_cap) c = (unsigned long long)e.hist_cap;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < c;
         k += (unsigned long long)gridDim.x * blockDim.x) {
      const uint32_t ent = e.hist[slot * (unsigned long long)e.hist_cap + k];
      const int64_t gidx = (int64_t)(ent & 0x7FFFFFFFu);
      const int inst = e.n_inst == 1 ? 0 : e.tile_info[gidx / kTile].x;
      if (inst < 0) continue;
      const InstDesc& dd = e.insts[inst];
      const int64_t j = gidx - dd.base;
      ev += (unsigned long long)(dd.row_ptr[j + 1] - dd.row_ptr[j]);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ev += __shfl_down_sync(kFull, ev, o);
  if ((threadIdx.x & 31) == 0 && ev) atomicAdd(out, ev);
}

__global__ void k_max_reduce(const int32_t* __restrict__ a, int64_t n, unsigned* out) {
  unsigned m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned)a[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

int g_deliver_grid = 0;

}  // namespace

void launch_init_state(const EngineDev& e, int inst, int n_tiles_inst, int first_tile,
                       cudaStream_t s) {
  if (n_tiles_inst > 0) k_init_state<<<n_tiles_inst, kUpdThreads, 0, s>>>(e, inst, first_tile);
}

void launch_update(const EngineDev& e, StepRef sr, cudaStream_t s) {
  if (e.four) {
    if (e.any_ext) k_update<true, true><<<e.n_tiles, kUpdThreads, 0, s>>>(e, sr);
    else k_update<false, true><<<e.n_tiles, kUpdThreads, 0, s>>>(e, sr);
  } else {
    if (e.any_ext) k_update<true, false><<<e.n_tiles, kUpdThreads, 0, s>>>(e, sr);
    else k_update<false, false><<<e.n_tiles, kUpdThreads, 0, s>>>(e, sr);
  }
}

void launch_close(const EngineDev& e, unsigned long long g, cudaStream_t s) {
  const int blocks = (e.total_R + 127) / 128;
  k_close<<<blocks > 0 ? blocks : 1, 128, 0, s>>>(e, g);
}

void launch_set_base(unsigned long long* base, unsigned long long g, cudaStream_t s) {
  k_set_base<<<1, 1, 0, s>>>(base, g);
}

int deliver_grid() {
  if (g_deliver_grid == 0) {
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_deliver<false, true>, kDelThreads, 0);
    if (occ < 1) occ = 1;
    g_deliver_grid = sms * occ;
  }
  return g_deliver_grid;
}

void launch_deliver(const EngineDev& e, int grid, StepRef sr, cudaStream_t s, int part) {
  if (grid < 2) grid = 2;  // with a segment ring, block 0 may take no items
  if (e.n_inst == 1) {
    if (e.four) k_deliver<true, true><<<grid, kDelThreads, 0, s>>>(e, sr, part);
    else k_deliver<false, true><<<grid, kDelThreads, 0, s>>>(e, sr, part);
  } else {
    if (e.four) k_deliver<true, false><<<grid, kDelThreads, 0, s>>>(e, sr, part);
    else k_deliver<false, false><<<grid, kDelThreads, 0, s>>>(e, sr, part);
  }
}

int persist_max_grid(const EngineDev& e) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* f = e.four ? (e.any_ext ? (const void*)k_persist<true, true, false>
                                      : (const void*)k_persist<false, true, false>)
                         : (e.any_ext ? (const void*)k_persist<true, false, false>
                                      : (const void*)k_persist<false, false, false>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kDelThreads, 0) != cudaSuccess) return 0;
  return sms * occ;
}

template <bool EXT, bool FOUR, bool SINGLE>
static cudaError_t coop_persist(const EngineDev& e, int grid, unsigned long long g0, int nsteps,
                                unsigned* count, unsigned long long limit_ns, cudaStream_t s) {
  EngineDev ea = e;
  void* args[] = {&ea, &g0, &nsteps, &count, &limit_ns};
  return cudaLaunchCooperativeKernel(k_persist<EXT, FOUR, SINGLE>, dim3(grid), dim3(kDelThreads),
                                     args, 0, s);
}

cudaError_t launch_persist(const EngineDev& e, int grid, unsigned long long g0, int nsteps,
                           unsigned* count, unsigned long long limit_ns, cudaStream_t s) {
  if (grid < 2) grid = 2;  // with a segment ring, block 0 may take no items
  cudaError_t r = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
  if (r != cudaSuccess) return r;
  const bool one = e.n_inst == 1;
  if (e.four) {
    if (e.any_ext)
      return one ? coop_persist<true, true, true>(e, grid, g0, nsteps, count, limit_ns, s)
                 : coop_persist<true, true, false>(e, grid, g0, nsteps, count, limit_ns, s);
    return one ? coop_persist<false, true, true>(e, grid, g0, nsteps, count, limit_ns, s)
               : coop_persist<false, true, false>(e, grid, g0, nsteps, count, limit_ns, s);
  }
  if (e.any_ext)
    return one ? coop_persist<true, false, true>(e, grid, g0, nsteps, count, limit_ns, s)
               : coop_persist<true, false, false>(e, grid, g0, nsteps, count, limit_ns, s);
  return one ? coop_persist<false, false, true>(e, grid, g0, nsteps, count, limit_ns, s)
             : coop_persist<false, false, false>(e, grid, g0, nsteps, count, limit_ns, s);
}

cudaError_t launch_barrier_probe(int grid, unsigned extra, int rounds, unsigned long long limit_ns,
                                 unsigned* count, unsigned* flags, cudaStream_t s) {
  cudaError_t r = cudaMemsetAsync(count, 0, sizeof(unsigned), s);
  if (r != cudaSuccess) return r;
  void* args[] = {&count, &extra, &rounds, &limit_ns, &flags};
  return cudaLaunchCooperativeKernel(k_barrier_probe, dim3(grid), dim3(32), args, 0, s);
}

void launch_ingest(int32_t N, int32_t j0, int32_t j1, int64_t e_base, const int64_t* row_ptr,
                   const int32_t* col_in, const void* w_in, const void* w2_in, int32_t w_dtype,
                   const uint8_t* delay_in, uint16_t* rec, int32_t dmax, int32_t seg_stride,
                   void* seg, int32_t seg_kind, int32_t* indeg, unsigned* wmax_bits, unsigned* err,
                   cudaStream_t s) {
  int64_t blocks = ((int64_t)(j1 - j0) * 32 + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  k_ingest<<<(int)blocks, 256, 0, s>>>(N, j0, j1, e_base, row_ptr, col_in, w_in, w2_in, w_dtype,
                                       delay_in, rec, dmax, seg_stride, seg, seg_kind, indeg,
                                       wmax_bits, err);
}

void launch_pending_events(const EngineDev& e, unsigned long long g, unsigned long long* out,
                           cudaStream_t s) {
  if (g == 0) return;
  const long long r0 = (long long)g - 1, r1 = (long long)g - 1 + e.bin_lead;
  k_pending_events<<<152, 256, 0, s>>>(e, r0, r1, out);
}

void launch_max_reduce(const int32_t* a, int64_t n, unsigned* out, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_max_reduce<<<(int)blocks, 256, 0, s>>>(a, n, out);
}


}  // namespace dbn

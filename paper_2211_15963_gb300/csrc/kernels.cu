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
  // channels
  const int words = e.four ? 4 : 2;
  for (int k = 0; k < words; ++k)
    *reinterpret_cast<int4*>(e.acc + (e.four ? 2 : 1) * gi0 + 2 * k) = make_int4(0, 0, 0, 0);
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
template <bool EXT, bool FOUR>
__global__ void __launch_bounds__(kUpdThreads, 4) k_update(EngineDev e, StepRef sr) {
  __shared__ RegionConst s_rc[kTileRegions];
  __shared__ uint32_t s_wtot[kUpdThreads / 32];
  __shared__ uint32_t s_hbase;
  __shared__ unsigned long long s_rbase;
  const int tile = blockIdx.x;
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
  // thread's four neurons
  int4 A[4];
  if (FOUR) {
#pragma unroll
    for (int k = 0; k < 4; ++k) A[k] = *reinterpret_cast<const int4*>(e.acc + 2 * gi0 + 2 * k);
  } else {
    const int4 a01 = *reinterpret_cast<const int4*>(e.acc + gi0);
    const int4 a23 = *reinterpret_cast<const int4*>(e.acc + gi0 + 2);
    A[0] = make_int4(a01.x, a01.x, a01.y, a01.y);
    A[1] = make_int4(a01.z, a01.z, a01.w, a01.w);
    A[2] = make_int4(a23.x, a23.x, a23.y, a23.y);
    A[3] = make_int4(a23.z, a23.z, a23.w, a23.w);
  }

  const int4 ti = e.tile_info[tile];  // instance, first region, regions touched
  const unsigned long long g = step_of(sr);
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
      *reinterpret_cast<int4*>(e.acc + (FOUR ? 2 : 1) * gi0 + 2 * k) = make_int4(0, 0, 0, 0);
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
  const int slot = (int)(g % (unsigned long long)e.D);
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

// FOUR: the engine keeps four accumulator channels per neuron; an edge adds
// its two weights (the one weight twice for one-weight records) to the
// channel pair of the source's class with one 64-bit atomic.  Every channel
// sum stays below 2^31 (the fixed-point scale is chosen so), so the low word
// never carries into the high one.
template <bool FOUR>
__global__ void __launch_bounds__(kDelThreads) k_deliver(EngineDev e, StepRef sr) {
  __shared__ unsigned long long s_pre[256];  // items whose delay is below index + 1
  __shared__ unsigned long long s_wsum[kDelThreads / 32];
  __shared__ unsigned long long s_total;
  const unsigned long long g = step_of(sr);
  const int D = e.D;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  // close the bin that ended with the previous iteration, one region per thread
  for (int gr = gtid; gr < e.total_R; gr += gridDim.x * blockDim.x) close_region(e, gr, g);
  // the slot this iteration's update will fill was last read by the previous one
  if (gtid == 0) e.hcount[g % (unsigned long long)D] = 0u;
  // The leading nA blocks copy the row start and segment counts of the
  // previous step's spikes into the delay-major ring (thread per spike, so
  // each store of a delay plane is coalesced across the warp) and take no
  // items; nA follows that step's spike count, the same in every block.
  unsigned long long c1 = 0;
  int nA = 0;
  const unsigned long long s1 = (g + (unsigned long long)D - 1ull) % (unsigned long long)D;
  if (e.seg_cap > 0 && g >= 1ull) {
    c1 = e.hcount[s1];
    if (c1 > (unsigned long long)e.hist_cap) c1 = (unsigned long long)e.hist_cap;
    if (c1 > (unsigned long long)e.seg_cap) c1 = (unsigned long long)e.seg_cap;
    const unsigned long long want = (c1 + kDelThreads - 1) / kDelThreads;
    const int most = gridDim.x >= 16 ? (int)gridDim.x / 8 : 1;  // the host launches >= 2 blocks
    nA = want < (unsigned long long)most ? (int)want : most;
  }
  if ((int)blockIdx.x < nA) {
    const size_t cap = (size_t)e.seg_cap;
    for (unsigned long long k = gtid; k < c1; k += (unsigned long long)nA * kDelThreads) {
      const uint32_t ent = e.hist[s1 * (unsigned long long)e.hist_cap + k];
      const int64_t gidx = (int64_t)(ent & 0x7FFFFFFFu);
      const int inst = e.n_inst == 1 ? 0 : e.tile_info[gidx / kTile].x;
      if (inst < 0) continue;  // never for a listed spike: tiles are reused D steps late
      const InstDesc& dd = e.insts[inst];
      if (dd.seg_kind != kSeg16) continue;
      const int64_t j = gidx - dd.base;
      e.hr0[s1 * cap + k] = __ldg(dd.row_ptr + j);
      const uint4* T = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(dd.seg) +
                                                      j * dd.seg_stride);
      uint16_t* H = e.hseg + (s1 * (size_t)e.dcap) * cap + k;
      const int nq = (dd.dmax + 7) >> 3;
      for (int q0 = 0; q0 < nq; q0 += 4) {
        uint4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = q0 + i < nq ? __ldg(T + q0 + i) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t wd[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int dl = (q0 + i) * 8 + u;
            if (dl < dd.dmax) H[(size_t)dl * cap] = (uint16_t)(wd[u >> 1] >> ((u & 1) * 16));
          }
        }
      }
    }
    return;
  }
  const int bB = (int)blockIdx.x - nA, nB = (int)gridDim.x - nA;  // item blocks

  // spikes of step g - d for d = threadIdx.x + 1, and their exclusive prefix
  unsigned long long c = 0;
  const int dme = threadIdx.x + 1;
  if (dme < D && g >= (unsigned long long)dme) {
    const unsigned long long h = e.hcount[(g - dme) % (unsigned long long)D];
    c = h < (unsigned long long)e.hist_cap ? h : (unsigned long long)e.hist_cap;
  }
  unsigned long long incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long acc = 0;
    for (int w = 0; w < kDelThreads / 32; ++w) {
      const unsigned long long t = s_wsum[w];
      s_wsum[w] = acc;
      acc += t;
    }
    s_total = acc;
  }
  __syncthreads();
  s_pre[threadIdx.x] = s_wsum[warp] + incl - c;
  const int nd = D - 1 < kDelThreads ? D - 1 : kDelThreads;  // delay buckets d = 1..nd
  const unsigned long long W = s_total;
  __syncthreads();

  unsigned long long ev = 0;
  const unsigned long long wstride = (unsigned long long)nB * blockDim.x;
  const unsigned long long wbase = (unsigned long long)bB * blockDim.x + warp * 32;
  for (unsigned long long b0 = wbase; b0 < W; b0 += wstride) {  // warp-uniform
    // each lane resolves one item: (spike, delay) -> its edge segment
    const unsigned long long t = b0 + lane;
    int64_t e0 = 0;
    uint32_t nseg = 0;
    int inst = 0;
    uint32_t cls = 0;
    if (t < W) {
      // bucket: the largest i with s_pre[i] <= t; delay d = i + 1
      int lo = 0, hi = nd - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pre[mid] <= t) lo = mid; else hi = mid - 1;
      }
      uint32_t d = (uint32_t)lo + 1u;
      const unsigned long long k = t - s_pre[lo];
      const unsigned long long slot = (g - d) % (unsigned long long)D;
      const uint32_t ent = e.hist[slot * (unsigned long long)e.hist_cap + k];
      const int64_t gidx = (int64_t)(ent & 0x7FFFFFFFu);
      cls = ent >> 31;
      inst = e.n_inst == 1 ? 0 : e.tile_info[gidx / kTile].x;
      if (inst < 0) inst = 0, d = 0u;  // (as above) -- takes no edges
      const InstDesc& dd = e.insts[inst];
      if (d >= 1u && (int32_t)d <= dd.dmax) {
        const int64_t j = gidx - dd.base;
        int64_t r0, a, b;
        if (dd.seg_kind == kSeg16 && d >= 2u && k < (unsigned long long)e.seg_cap) {
          // from the delay-major ring (consecutive lanes, consecutive spikes)
          const size_t cap = (size_t)e.seg_cap;
          r0 = __ldg(e.hr0 + slot * cap + k);
          const uint16_t* H = e.hseg + (slot * (size_t)e.dcap) * cap + k;
          a = (int64_t)__ldg(H + (size_t)(d - 2u) * cap);
          b = (int64_t)__ldg(H + (size_t)(d - 1u) * cap);
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
      }
    }
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
    for (uint32_t f = 0; f < total; f += 32) {  // warp-uniform
      const uint32_t fi = f + lane;
      int L = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int cand = L + step < 32 ? L + step : 31;
        const uint32_t v = __shfl_sync(kFull, ex, cand);
        if (L + step < 32 && v <= fi) L = cand;
      }
      const int64_t q0 = __shfl_sync(kFull, e0, L);
      const uint32_t qx = __shfl_sync(kFull, ex, L);
      const int qi = __shfl_sync(kFull, inst, L);
      const uint32_t qc = __shfl_sync(kFull, cls, L);
      if (fi < total) {
        const InstDesc& dd = e.insts[qi];
        const int64_t ei = q0 + (int64_t)(fi - qx);
        uint32_t tg, wb, wb2 = 0;
        if (FOUR && dd.two_w) {  // 8-byte record: target, weight | second weight << 16
          const uint2 r4 = __ldg(reinterpret_cast<const uint2*>(dd.rec) + ei);
          tg = r4.x;
          wb = r4.y & 0xFFFFu;
          wb2 = r4.y >> 16;
        } else if (dd.rec) {
          const uint16_t* r3 = dd.rec + 3 * ei;
          tg = (uint32_t)__ldg(r3) | ((uint32_t)__ldg(r3 + 1) << 16);
          wb = __ldg(r3 + 2);
          wb2 = wb;
        } else {
          tg = __ldg(dd.col + ei) & dd.tmask;
          wb = __ldg(dd.w + ei);
          wb2 = wb;
        }
        const int q = __float2int_rn(__fmul_rn(__uint_as_float(wb << 16), dd.two_S));
        if (FOUR) {
          const int q2 = __float2int_rn(__fmul_rn(__uint_as_float(wb2 << 16), dd.two_S));
          unsigned long long* accp = reinterpret_cast<unsigned long long*>(e.acc) +
                                     2 * (size_t)(dd.base + (int64_t)tg) + qc;
          atomicAdd(accp, ((unsigned long long)(uint32_t)q2 << 32) | (uint32_t)q);
        } else {
          int* accp = reinterpret_cast<int*>(e.acc + dd.base) + qc;
          atomicAdd(accp + 2 * (size_t)tg, q);
        }
      }
    }
    if (lane == 0) ev += total;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ev += __shfl_down_sync(kFull, ev, o);
  __syncthreads();
  if (lane == 0) s_wsum[warp] = ev;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < kDelThreads / 32; ++w) s += s_wsum[w];
    if (s) atomicAdd(e.events, s);
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_deliver<false>, kDelThreads, 0);
    if (occ < 1) occ = 1;
    g_deliver_grid = sms * occ;
  }
  return g_deliver_grid;
}

void launch_deliver(const EngineDev& e, int grid, StepRef sr, cudaStream_t s) {
  if (grid < 2) grid = 2;  // with a segment ring, block 0 may take no items
  if (e.four) k_deliver<true><<<grid, kDelThreads, 0, s>>>(e, sr);
  else k_deliver<false><<<grid, kDelThreads, 0, s>>>(e, sr);
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

void launch_max_reduce(const int32_t* a, int64_t n, unsigned* out, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_max_reduce<<<(int)blocks, 256, 0, s>>>(a, n, out);
}


}  // namespace dbn

/*
 * dbnet -- GB300 (sm_103a) library for the hot path of the Digital Brain:
 * conductance leaky integrate-and-fire networks with delayed spike delivery,
 * the regional Balloon-Windkessel BOLD readout, and the diffusion ensemble
 * Kalman filter of hierarchical mesoscale data assimilation (HMDA).
 *
 * Conventions shared by every entry point
 *   - Status: every int-returning call returns DBNET_OK (0) or a negative
 *     DBNET_E* code; dbnet_strerror() names it and dbnet_last_error() gives
 *     the detail of the most recent failure on the calling thread.  After a
 *     CUDA failure a handle is poisoned: later calls return DBNET_ESTATE.
 *   - Ownership: input arrays are caller-owned host memory, read (copied) at
 *     the call and never retained.  Device state is owned by the handle and
 *     freed by the matching *_destroy.  Output arrays are caller-allocated
 *     host memory.
 *   - Streams: all device work is enqueued on the CUDA stream given at
 *     create (NULL = a non-blocking stream the handle creates and owns);
 *     step calls return without waiting, read calls synchronise that stream
 *     first.
 *   - Threads: a handle must not be used from two threads at once.
 *   - Units: mV, ms, nF, microsiemens, nA; BOLD model constants in seconds.
 *   - Neuron numbering: neurons are sorted by region; inside a region the
 *     excitatory neurons come first.  Spikes of excitatory sources drive the
 *     AMPA and NMDA channels of their targets, inhibitory ones GABA_A and
 *     GABA_B (Extended Data Table 2, "Synapse model").
 */
#ifndef DBNET_H
#define DBNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DBNET_OK 0
#define DBNET_EINVAL (-1)      /* malformed graph, parameters or arguments */
#define DBNET_ENOMEM (-2)      /* device or host allocation failed */
#define DBNET_ECUDA (-3)       /* a CUDA runtime call failed */
#define DBNET_ETIMEOUT (-4)    /* a grid barrier of the persistent stepper
                                  waited longer than its limit (1 s); the
                                  handle is then poisoned */
#define DBNET_EOVERFLOW (-5)   /* fixed-point accumulation could overflow int32 */
#define DBNET_ESTATE (-6)      /* handle poisoned by an earlier failure */
#define DBNET_ERANGE (-7)      /* a caller buffer or a fixed capacity is too small */
#define DBNET_EUNSUPPORTED (-8)

#define DBNET_WEIGHT_F32 0
#define DBNET_WEIGHT_BF16 1

#define DBNET_SCHEDULE_AUTO 0
#define DBNET_SCHEDULE_SEQUENTIAL 1
#define DBNET_SCHEDULE_PIPELINED 2
#define DBNET_SCHEDULE_PERSISTENT 3

typedef struct dbnet dbnet_t;
typedef struct dbens dbens_t;

/* Network graph: CSR by source (the paper's connection table, Supplementary
 * Table 5, transposed so that a spiking neuron finds its out-edges; push
 * delivery, Supplementary Algorithm 2).
 *   n_neurons        N, 1 <= N < 2^31
 *   n_regions        R >= 1
 *   region_offsets   [R+1] int32, 0 = offsets[0] < ... < offsets[R] = N
 *   n_exc            [R] int32, excitatory neurons at the start of region r
 *   row_ptr          [N+1] int64, row_ptr[0] = 0, non-decreasing
 *   col              [E] int32 target index, 0 <= col < N
 *   weight           [E] non-negative synaptic weight w, as float32 or as
 *                    BF16 bit patterns (weight_dtype); stored as BF16
 *                    (round to nearest even) on the device
 *   delay            [E] uint8 delay in steps, 1..255; within each row the
 *                    delays must be non-decreasing
 *   weight2          NULL: one weight per edge, shared by both channels of
 *                    the source's class (AMPA and NMDA for an excitatory
 *                    source, GABA_A and GABA_B for an inhibitory one).
 *                    Otherwise [E] a second weight per edge, same dtype and
 *                    rules as weight (the connection table of
 *                    Supplementary Table 5 holds one weight per channel):
 *                    weight then feeds AMPA / GABA_A and weight2 NMDA /
 *                    GABA_B, and the engine keeps four accumulator channels
 *                    per neuron instead of two.  Zero-initialised callers get
 *                    NULL.
 * A spike of source j at step n reaches target col[e] through edge e in the
 * accumulator consumed at step n + delay[e].  Violations give DBNET_EINVAL. */
typedef struct {
  int32_t n_neurons;
  int32_t n_regions;
  const int32_t* region_offsets;
  const int32_t* n_exc;
  const int64_t* row_ptr;
  const int32_t* col;
  const void* weight;
  int32_t weight_dtype;
  const uint8_t* delay;
  const void* weight2;
} dbnet_graph_t;

/* Per-region neuron and synapse constants (the property table of
 * Supplementary Table 5, one row per region).  Channels u = AMPA, NMDA,
 * GABA_A, GABA_B.
 *   C, gL, VL, Vth, Vreset, Tref   membrane (Methods, capacitance-voltage eq.)
 *   Vu[u], tau_u[u], g_u[u]        reversal potential, trace decay time and
 *                                  maximal conductance (Methods, Eq. 2)
 *   I_ext                          constant injected current
 *   drive_rate_hz, drive_K, w_ext  Poisson background: drive_K independent
 *                                  sources of rate drive_rate_hz per neuron,
 *                                  each event adding w_ext to the excitatory
 *                                  traces (Extended Data Table 2, "Input")
 *   ou_mu, ou_sigma, ou_tau        background current I_bg, an Ornstein-
 *                                  Uhlenbeck process per neuron (Methods,
 *                                  Eq. 1; Extended Data Table 2, "OU current":
 *                                  0.66, 0.12, 10 ms), integrated by Euler-
 *                                  Maruyama: I_bg += (mu - I_bg) dt/tau +
 *                                  sigma sqrt(2 dt/tau) xi, xi standard normal
 *                                  (Box-Muller of Philox stream 4, FP32 on the
 *                                  device); added after I_ext inside the dt/C
 *                                  bracket with its value before the step; it
 *                                  starts at mu.  Off when ou_mu = ou_sigma = 0;
 *                                  else ou_tau > 0 and ou_sigma >= 0.
 *   iext_shape                     > 0: heterogeneous injected current (Methods:
 *                                  I_ext,i Gamma distributed): neuron i receives
 *                                  I_ext * G_i / k, G_i ~ Gamma(k = iext_shape, 1)
 *                                  drawn once at create (Marsaglia-Tsang on its
 *                                  Philox words of stream 5, FP64); 0: I_ext. */
typedef struct {
  double C, gL, VL, Vth, Vreset, Tref;
  double Vu[4], tau_u[4], g_u[4];
  double I_ext, drive_rate_hz, drive_K, w_ext;
  double ou_mu, ou_sigma, ou_tau;
  double iext_shape;
} dbnet_region_params_t;

/* Run options.
 *   dt_ms            Euler step (Supplementary Sec. 3: 0.1 or 1 ms)
 *   bin_ms           neural-activity bin that feeds the BOLD model; a whole
 *                    number of steps
 *   tr_ms            BOLD sampling period (800 ms in the paper); a whole
 *                    number of bins
 *   z_scale          z = z_scale * (spikes of the region in the bin) / size
 *   bw_*             Balloon-Windkessel constants (Extended Data Table 4)
 *   seed, net_id     Philox4x64-10 key; the drive and the initial state of
 *                    neuron i at step n use counter (n, i/4, stream, 0)
 *   fixed_shift      S of the fixed-point accumulators q(w) = rint(w 2^S);
 *                    0 = automatic (16, lowered until one step's worst-case
 *                    arrivals fit int32)
 *   precision        32 (FP32 state; the only mode the device path runs)
 *   raster_capacity  spikes kept for dbnet_read_spikes (0 = none)
 *   bold_capacity    BOLD samples kept per region
 *   autotune_at      step at which the delivery is tuned (-1 = never): with an
 *                    automatic emit_delay candidate, first D + 64 steps
 *                    without and D + 64 with it, the last 64 of each timed,
 *                    the faster kept; then every launch shape -- a delivery
 *                    grid (1..4 blocks per SM, and for networks of at most
 *                    two 1,024-neuron tiles per SM also an eighth, a quarter
 *                    and half of the SMs) on each schedule the schedule
 *                    option admits (the persistent one only while its blocks
 *                    hold at most one tile each) -- runs 64 steps timed by
 *                    CUDA events, three times each in turn (after the first
 *                    round those over twice the best drop out), and the
 *                    smallest total is kept.
 *                    Results depend on none of these choices (integer
 *                    accumulation).  Default 2000 (200 ms at dt 0.1 ms, past
 *                    the onset).
 *   bin_spikes       1: spikes are handed on at bin edges (Supplementary Sec. 3,
 *                    "Numerical method": the accumulated spike A_j(t) is non-
 *                    zero only at t = k * bin and marks a spike of j in
 *                    (t - bin, t]).  A spike emitted in any step of bin
 *                    [k spb, (k+1) spb) (spb = bin_ms / dt_ms) reaches the
 *                    targets of its delay-d edges at step (k+1) spb - 1 + d;
 *                    d = 1 is the paper's scheme.  Needs T_ref >= bin_ms -
 *                    dt_ms in every region (so a neuron fires at most once
 *                    per bin and A_j is 0 or 1; else DBNET_EINVAL) and
 *                    longest delay + spb <= 256.  0 (default): every spike
 *                    is handed on in its own step.
 *   emit_delay       which delays are added at emission instead of when they
 *                    come due (the results are the same: the accumulators
 *                    are exact integers).  Arrival time reads each due
 *                    (spike, delay) segment of a row on its own, which pays
 *                    when segments are long; at emission the accumulators
 *                    form a ring of D slots (D x N x 8 bytes, taken only when
 *                    it fits a third of the free device memory) and a
 *                    spike's edges of delay >= emit_delay go straight into
 *                    the slot of their arrival step, its short segments read
 *                    in one pass.  -1 (default): none; d >= 1: delays >= d;
 *                    0: the delays from which every (row, delay) segment
 *                    holds fewer than 4 edges on average (estimated from a
 *                    sample of rows at create), kept only if the autotuner
 *                    measures it faster than none.  Request servers use none.
 *                    On the benchmark networks (in-degree 1,000, 1.3 edges
 *                    per cross-region delay) emission measured slower: its
 *                    scattered additions land in a ring far larger than the
 *                    L2.
 *   schedule         how a step's two kernels are ordered (the results are
 *                    the same): DBNET_SCHEDULE_SEQUENTIAL, the delivery of
 *                    step n then its update; DBNET_SCHEDULE_PIPELINED, the
 *                    delivery of step n + 1's delays >= 2 (which need only
 *                    spikes of steps <= n - 1) on a second stream beside the
 *                    update of step n, so that the latency-bound delivery
 *                    runs under the bandwidth-bound update, then the rest of
 *                    step n + 1's delivery; DBNET_SCHEDULE_PERSISTENT, many
 *                    steps in one cooperative launch (the same delivery and
 *                    update device code, separated by grid barriers whose
 *                    waits give up after 1 s with DBNET_ETIMEOUT), which
 *                    saves the two launches per step where a step's kernels
 *                    are short; DBNET_SCHEDULE_AUTO (default): sequential
 *                    until the autotuner times all three.
 *   deliver_blocks   blocks of the delivery grid (>= 2; on the persistent
 *                    schedule at most the co-resident blocks, else
 *                    DBNET_EINVAL at the first step), and the autotuner then
 *                    tunes only the schedule; 0 (default): 1 to 4 blocks
 *                    per SM, as the occupancy allows, until the autotuner
 *                    picks one. */
typedef struct {
  double dt_ms, bin_ms, tr_ms, z_scale;
  double bw_kappa, bw_gamma, bw_tau, bw_alpha, bw_rho, bw_V0;
  uint64_t seed, net_id;
  int32_t fixed_shift;
  int32_t precision;
  int64_t raster_capacity;
  int64_t bold_capacity;
  int64_t autotune_at;
  int32_t bin_spikes;
  int32_t emit_delay;
  int32_t schedule;
  int32_t deliver_blocks;
} dbnet_options_t;

typedef struct {
  int64_t step;              /* steps completed */
  int64_t spikes;            /* spikes emitted */
  int64_t events;            /* synaptic events: the out-degree of every spike
                                handed on so far (whichever later step adds each
                                edge), by the engine behind the handle (for an
                                ensemble member: the whole ensemble) */
  int64_t raster_len;        /* spikes recorded */
  int64_t raster_dropped;    /* spikes not recorded for lack of capacity */
  int64_t bold_samples;      /* BOLD samples recorded */
  int32_t fixed_shift;       /* S in use */
  int32_t max_delay;         /* longest delay of the graph, steps */
  int32_t packed_edges;      /* 1: edges held as 6-byte (target, BF16 weight)
                                records, 8-byte (target, two BF16 weights) with
                                two weights per edge */
  int32_t weights_rounded;   /* 1 when some float32 weight was not a BF16 value */
  int32_t deliver_blocks;    /* delivery grid in use */
  int32_t autotuned;         /* 1 once the autotuner has chosen that grid */
  int32_t two_weights;       /* 1: four accumulator channels (two weights per edge) */
  int32_t seg_ring;          /* spikes per step whose segments the delivery reads
                                from its delay-major ring; a step's later spikes
                                (and graphs with u32 segment tables) are resolved
                                from the graph's own tables */
  int32_t emit_delay;        /* delays >= this are added at emission (0: none) */
  int32_t schedule;          /* DBNET_SCHEDULE_SEQUENTIAL, _PIPELINED or
                                _PERSISTENT: the schedule in use */
} dbnet_stats_t;

/* Name of a status code (static string). */
const char* dbnet_strerror(int code);

/* Optional device allocator.  By default every handle takes its device
 * memory with cudaMalloc and returns it with cudaFree.  A caller that owns a
 * memory pool -- PyTorch's caching allocator, for instance -- installs an
 * allocator here, and every device allocation of handles created afterwards
 * (network state, graph records, rings, ensemble and server buffers, the
 * server's arena) comes from alloc and goes back to free:
 *   alloc(bytes, stream, ctx)   returns device memory of at least bytes,
 *                               aligned to 256 bytes, or NULL (the call that
 *                               needed it then fails with DBNET_ENOMEM);
 *                               stream is the cuda_stream given to the create
 *                               call (NULL: the legacy default stream)
 *   free(ptr, bytes, stream, ctx) returns it; the handle's stream has been
 *                               synchronised first, so the memory is idle.
 * Each allocation goes back to the allocator it came from, so installing
 * another (or NULL, which restores cudaMalloc) affects only later handles;
 * the functions and ctx must stay valid until those handles are destroyed.
 * Process-wide; install it before creating handles, not while another
 * thread creates one.  The allocation-free entry point never calls it.
 * (The paper has no counterpart: this serves embedding in a host framework.) */
typedef void* (*dbnet_alloc_fn)(size_t bytes, void* cuda_stream, void* ctx);
typedef void (*dbnet_free_fn)(void* ptr, size_t bytes, void* cuda_stream, void* ctx);
typedef struct {
  dbnet_alloc_fn alloc;
  dbnet_free_fn free;
  void* ctx;
} dbnet_allocator_t;
/* a NULL allocator, or one with NULL functions, restores cudaMalloc */
int dbnet_set_allocator(const dbnet_allocator_t* allocator);

/* Detail of the last failure on the calling thread (static per thread). */
const char* dbnet_last_error(void);

/* sizeof of the public structs, for bindings to check their layouts:
 * out[0..10] = dbnet_graph_t, dbnet_region_params_t, dbnet_options_t,
 * dbnet_stats_t, dbens_enkf_t, dbnet_device_graph_t, dbsrv_options_t,
 * dbsrv_request_t, dbsrv_status_t, dbsrv_stats_t, 0 (reserved).  Writes
 * min(n, 11) entries; returns the number of structs (10).  Needs no GPU. */
int dbnet_abi_sizes(int64_t* out, int n);

/* Fill *o with the defaults: dt 0.1 ms, bin 1 ms, TR 800 ms, z_scale 1,
 * the standard hemodynamic constants, seed 1, net_id 0, automatic S,
 * precision 32, no raster, 4096 BOLD samples, autotune at step 2000, no
 * spike binning, no emission-time delivery. */
int dbnet_options_default(dbnet_options_t* o);

/* Build a network on the current CUDA device (Methods, "Constructing the
 * Digital Brain model": the neurons with their property table and the
 * connection table of Supplementary Table 5, here one network on one GPU):
 * copy the graph and parameters (edges in chunks of rows through staging
 * buffers), validate them on the device, store the edges as 6-byte
 * (target, BF16 weight) records, choose S and set the initial state (V
 * uniform in [V_reset, V_th) from Philox stream 1, which desynchronises the
 * neurons as the paper's initial background spikes do, Supplementary Sec. 3;
 * traces zero).  Also builds the per-row delay-segment table
 * (N x longest delay counts, u16 when every row has < 65536 edges).
 * params: [n_regions].  cuda_stream: a cudaStream_t or NULL.
 * Returns DBNET_EINVAL for a malformed graph or parameter set,
 * DBNET_EOVERFLOW when the chosen S could overflow, DBNET_ENOMEM, DBNET_ECUDA. */
int dbnet_create(const dbnet_graph_t* graph, const dbnet_region_params_t* params,
                 const dbnet_options_t* options, void* cuda_stream, dbnet_t** out);

/* Advance by n_steps Euler steps (Supplementary Sec. 3, Eqs. 3 and 5; push
 * delivery, Supplementary Algorithm 2; BOLD per bin, Extended Data Table 4).
 * Enqueued on the handle's stream; returns without waiting. */
int dbnet_step(dbnet_t* h, int64_t n_steps);

/* Wait for the handle's stream. */
int dbnet_sync(dbnet_t* h);

/* Measurement form of dbnet_step: the same n_steps, but every kernel is
 * launched on its own (no graph replay) between CUDA events recorded on the
 * handle's stream.  Waits for completion, then ms[0] = summed device time of
 * the delivery kernel and ms[1] = of the neuron-update kernel over the
 * n_steps launches of each.  Results are identical to dbnet_step. */
int dbnet_step_timed(dbnet_t* h, int64_t n_steps, double* ms);

/* Recorded spikes with t0 <= step < t1, sorted by (step, id), written to
 * step[] and id[] (capacity cap): the spike trains the model outputs
 * (Results, "the output describing the action potentials over time";
 * Supplementary Algorithm 2's per-step list of spiking neurons).
 * *n_out = number written; DBNET_ERANGE when more than cap match (the first
 * cap are written).  A step is the Euler step at whose end V reached V_th. */
int dbnet_read_spikes(dbnet_t* h, int64_t t0, int64_t t1, int32_t* step, int32_t* id,
                      int64_t cap, int64_t* n_out);

/* BOLD samples y[k][r] (row-major, k-th TR), at most cap_samples rows: the
 * Balloon-Windkessel output of Extended Data Table 4 for each region,
 * sampled once per TR (800 ms in the paper's fMRI, Supplementary Sec. 1),
 * the observation HMDA assimilates (Supplementary Sec. 6). */
int dbnet_read_bold(dbnet_t* h, double* y, int64_t cap_samples, int64_t* n_out);

/* Hemodynamic state x[r][4] = (s, f, v, q) per region. */
int dbnet_read_bw(dbnet_t* h, double* x);

/* Neuron state: V[N], J[4][N] (channel-major), ref[N] (remaining refractory
 * steps).  Any pointer may be NULL. */
int dbnet_read_state(dbnet_t* h, float* V, float* J, int32_t* ref);

/* Overwrite the neuron state (same layout; NULL leaves a field unchanged).
 * ref values must lie in 0..255. */
int dbnet_set_state(dbnet_t* h, const float* V, const float* J, const int32_t* ref);

/* Background OU current I_bg[N] (zero in regions without it): read, or
 * overwrite before the next step. */
int dbnet_read_ibg(dbnet_t* h, float* I_bg);
int dbnet_set_ibg(dbnet_t* h, const float* I_bg);

/* Counters of the run: steps, spikes, synaptic events (every out-edge of
 * every spike handed on, as Supplementary Algorithm 2 pushes them; the
 * paper's throughput figures count the same events), raster and BOLD
 * lengths, and the shapes the engine chose. */
int dbnet_stats(dbnet_t* h, dbnet_stats_t* out);

void dbnet_destroy(dbnet_t* h);

/* Checks the grid barrier of the persistent stepper on the current device
 * (no counterpart in the paper): one cooperative launch of `blocks` blocks
 * (1 .. the number of SMs) passes `rounds` (>= 1) barriers, each of which
 * expects `missing` arrivals more than the grid makes.  With missing = 0
 * every barrier completes and the call returns DBNET_OK; with missing > 0
 * nothing makes the awaited arrivals, the first wait gives up after
 * limit_us microseconds (1 .. 10^7) of the device's global timer, every
 * block returns, and the call returns DBNET_ETIMEOUT with the device still
 * usable.  The call synchronises the device's default stream.  DBNET_EINVAL
 * for arguments outside those ranges. */
int dbnet_barrier_probe(int32_t blocks, int32_t missing, int32_t rounds, int64_t limit_us);

/* ---------------------------------------------------------------------------
 * Ensemble of networks for HMDA (Methods, "Statistical inference ... by
 * HMDA"; Supplementary Sec. 6 and Algorithm 3).  n_members networks share one
 * graph and differ in their per-region AMPA and GABA_A conductance scales
 * (the hyperparameters theta, held as natural logarithms) and in their
 * Philox key (net_id = options.net_id + member).  The analysis state of a
 * member is, per region r, the block (theta_AMPA, theta_GABA_A, s, f, v, q, y).
 * ------------------------------------------------------------------------ */
#define DBENS_DIFFUSION 0 /* one observer per region, fused with weight gamma */
#define DBENS_GLOBAL 1    /* one observer of all regions (textbook EnKF) */

/* What each of a region's two log scales multiplies (Supplementary Sec. 6:
 * the maximal conductances for resting-state data, the injected current for
 * task data).  A scale family keeps its shape under cdf^-1(cdf(.; old); new),
 * so the region's value is base * exp(theta). */
#define DBENS_T_DEFAULT 0 /* slot 0: g_AMPA, slot 1: g_GABA_A */
#define DBENS_T_AMPA 1
#define DBENS_T_NMDA 2
#define DBENS_T_GABA_A 3
#define DBENS_T_GABA_B 4
#define DBENS_T_IEXT 5    /* the region's injected current (task variant) */
#define DBENS_T_NONE (-1) /* carried in the state, scales nothing */

typedef struct {
  double obs_var;     /* Gamma_o: observation noise variance of every BOLD signal */
  double gamma;       /* fusion coefficient of Supplementary Algorithm 3 */
  double rw_sigma;    /* std of the random walk of theta per analysis */
  double theta_lo;    /* theta is kept in [theta_lo, theta_hi] */
  double theta_hi;
  double floor;       /* f, v, q are kept >= floor after an analysis */
  int32_t mode;       /* DBENS_DIFFUSION or DBENS_GLOBAL */
  int32_t target[2];  /* DBENS_T_* of the two log scales (two distinct targets) */
} dbens_enkf_t;

/* base: [R] parameters before scaling; log_scale_init: [M][R][2] initial
 * theta of the two targets.  Errors as dbnet_create. */
int ens_create(const dbnet_graph_t* graph, const dbnet_region_params_t* base,
               int32_t n_members, const double* log_scale_init,
               const dbnet_options_t* options, const dbens_enkf_t* enkf,
               void* cuda_stream, dbens_t** out);

/* Advance every member by n_steps (one batched launch sequence). */
int ens_step(dbens_t* h, int64_t n_steps);

/* One analysis at the current time (Supplementary Algorithm 3, steps 4-7, in
 * FP64 on the device) against y_obs[R], using each member's latest BOLD
 * sample, then the random walk of theta and the rescaling of the members'
 * conductances.  eps_obs [M][R] and xi_rw [M][R][2] are standard-normal draws
 * (NULL: drawn on the device from Philox).  y_pred_mean [R] (may be NULL)
 * receives the forecast ensemble mean of y before the analysis.
 * DBNET_EINVAL for a non-finite y_obs, eps_obs or xi_rw (checked on the
 * host) and for an analysis that fails on the device (a covariance that is
 * not positive definite, or a non-finite analysed state); a failed analysis
 * leaves theta, the hemodynamic state and the members' constants unchanged. */
int ens_assimilate(dbens_t* h, const double* y_obs, const double* eps_obs,
                   const double* xi_rw, double* y_pred_mean);

/* Member states: theta [M][R][2], bw [M][R][4], y [M][R] (latest sample).
 * Any pointer may be NULL. */
int ens_read(dbens_t* h, double* theta, double* bw, double* y);

/* Access to one member as a network view (reads only): the returned handle
 * is owned by the ensemble and valid until ens_destroy. */
int ens_member(dbens_t* h, int32_t member, dbnet_t** out);

void ens_destroy(dbens_t* h);

/* ---------------------------------------------------------------------------
 * Allocation-free run.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory once they are running --
 * for instance code inside a framework whose arena owns all device memory,
 * or a closed loop that must not pay cudaMalloc's implicit device-wide
 * synchronisation.  It performs no cudaMalloc, cudaFree or other allocating
 * call.  Its scratch (spike ring, accumulators, counters, region constants)
 * is one static device array of DBNET_NOALLOC_SCRATCH_BYTES that every GPU
 * loading this library holds until the process exits.
 *
 * Graph: row_ptr, col, weight_bf16 and delay are DEVICE arrays in the same
 * layout as dbnet_graph_t (delays non-decreasing within a row); they are
 * validated on the device and never modified.  region_offsets and n_exc are
 * HOST arrays.
 * Run: the network starts from the same initial state as dbnet_create (V
 * uniform in [V_reset, V_th) from Philox stream 1, traces zero, no spike in
 * flight) and advances n_steps exactly as dbnet_step does.
 * Outputs (DEVICE arrays owned by the caller): V[n_pad], J[4][n_pad]
 * (channel-major, row stride n_pad), ref[n_pad] (u8), with n_pad = N rounded
 * up to a multiple of 1024, each 16-byte aligned (else DBNET_EINVAL: whole
 * tiles move by bulk copies); raster_step/raster_id[raster_cap] receive the
 * spikes (unordered within a step; more than raster_cap are dropped and
 * counted).  *n_spikes and *n_events (host) receive the totals.
 * Limits: N <= DBNET_NOALLOC_MAX_NEURONS, R <= DBNET_NOALLOC_MAX_REGIONS and
 * n_pad * (longest delay + 1) <= DBNET_NOALLOC_MAX_LIVE (the spike ring);
 * larger inputs return DBNET_ERANGE.
 * Set-up: the first call on each device looks up the scratch address with
 * cudaGetSymbolAddress while that device is current; make that first call
 * before any stream capture.  The address is kept for the life of the
 * process, so the library must not be used across a cudaDeviceReset (or any
 * other destruction of the device's primary context).  The call waits for
 * its work to finish.
 * Every call reuses the same scratch and clears it first, so calls that
 * overlap on the GPU (from several threads or streams) race. */
#define DBNET_NOALLOC_MAX_NEURONS 65536
#define DBNET_NOALLOC_MAX_REGIONS 64
#define DBNET_NOALLOC_MAX_LIVE (1 << 22)
#define DBNET_NOALLOC_SCRATCH_BYTES (18u << 20)

typedef struct {
  int32_t n_neurons;
  int32_t n_regions;
  const int32_t* region_offsets; /* host [R+1] */
  const int32_t* n_exc;          /* host [R] */
  const int64_t* row_ptr;        /* device [N+1] */
  const int32_t* col;            /* device [E] */
  const uint16_t* weight_bf16;   /* device [E] */
  const uint8_t* delay;          /* device [E] */
} dbnet_device_graph_t;

int dbnet_run_noalloc(const dbnet_device_graph_t* graph, const dbnet_region_params_t* params,
                      const dbnet_options_t* options, int64_t n_steps, float* V, float* J,
                      uint8_t* ref, int32_t* raster_step, int32_t* raster_id,
                      int64_t raster_cap, int64_t* n_spikes, int64_t* n_events,
                      void* cuda_stream);

/* ---------------------------------------------------------------------
 * Request server: continuous batching of simulation requests on one GPU.
 *
 * The paper runs one brain model per machine; it has no request server.
 * This is the serving form of the same step: many independent networks
 * (requests) share one engine, and every update and delivery launch covers
 * all requests resident at that moment.  A request is admitted when a
 * request slot, contiguous neuron tiles, region slots and room in the
 * server's device arena are free; until then it waits in a queue (first
 * fit over the oldest queued requests).  Its state stays resident until it
 * has run its n_steps; its results are then copied to the host, and its
 * slot, tiles and memory return to the pool once D more iterations have
 * completed (no spike of it is still in flight).  Requests do not interact:
 * each gives the same spikes, state and BOLD as the same network created
 * alone with dbnet_create and the same seed, net_id and options.
 * All device memory of requests comes from one arena allocated at
 * dbsrv_create, so admission and retirement never allocate or free device
 * memory.  A handle is not thread-safe.
 * ------------------------------------------------------------------- */
typedef struct dbsrv dbsrv_t;

typedef struct {
  int64_t max_neurons;    /* neuron capacity (whole tiles of 1024) */
  int32_t max_requests;   /* request slots (running or cooling down) */
  int32_t max_regions;    /* region slots */
  int32_t max_delay;      /* longest delay any request may use, steps (1..255) */
  int32_t chunk_steps;    /* Euler steps per scheduling round */
  int64_t arena_bytes;    /* device memory for the requests' graphs and buffers */
  int32_t max_inflight;   /* rounds enqueued ahead of the host */
  int32_t two_weights;    /* 1: four accumulator channels per neuron, so that
                             requests may carry two weights per edge (8 more
                             bytes per neuron and step in the update); 0:
                             such a request fails with DBNET_EUNSUPPORTED */
  dbnet_options_t run;    /* dt, bin, TR, z_scale, hemodynamic constants,
                             fixed_shift, autotune_at, precision; seed, net_id
                             and capacities come with each request */
} dbsrv_options_t;

typedef struct {
  int64_t n_steps;        /* Euler steps to run (>= 1) */
  uint64_t seed, net_id;  /* Philox key, as in dbnet_options_t */
  uint64_t graph_key;     /* non-zero: requests with the same key share one
                             device copy of the graph (the caller asserts the
                             graphs are identical); 0: a private copy */
  int64_t bold_capacity;  /* BOLD samples kept; 0 = all of n_steps */
  int64_t raster_capacity;/* spikes kept (0 = none) */
} dbsrv_request_t;

#define DBSRV_QUEUED 0
#define DBSRV_RUNNING 1
#define DBSRV_DONE 2
#define DBSRV_FAILED 3

typedef struct {
  int32_t state;          /* DBSRV_* */
  int32_t error;          /* status code when FAILED */
  int64_t steps;          /* steps completed, as known to the host */
  int64_t spikes;         /* spikes emitted (final when DONE) */
  int64_t bold_samples;   /* BOLD samples held (when DONE) */
  int64_t raster_len;     /* spikes held (when DONE) */
  double queued_s;        /* submit -> admission (wall clock) */
  double run_s;           /* admission -> results on the host */
  double latency_s;       /* submit -> results on the host */
} dbsrv_status_t;

typedef struct {
  int64_t iterations;     /* engine iterations completed on the device */
  int64_t events;         /* synaptic events applied, all requests */
  int32_t running, queued, cooling, done;
  int64_t arena_used, arena_bytes;
  int32_t tiles_in_use, tile_extent;
} dbsrv_stats_t;

/* Defaults: 8,388,608 neurons, 64 requests, 1,024 regions, delays <= 255,
 * 256 steps per round, a 64 GiB arena, 2 rounds in flight,
 * dbnet_options_default() for the run options. */
int dbsrv_options_default(dbsrv_options_t* o);

/* Allocate the pool (neuron state, spike rings, arena) on the current
 * device.  cuda_stream: the stream every step runs on (NULL: its own).
 * DBNET_EINVAL for bad options, DBNET_ENOMEM when the pool does not fit. */
int dbsrv_create(const dbsrv_options_t* options, void* cuda_stream, dbsrv_t** out);

/* Queue a request.  graph and params follow dbnet_create; params [R].  The
 * graph's host arrays must stay valid until the request leaves the queue
 * (dbsrv_poll reports RUNNING, DONE or FAILED); params are copied now.
 * Host checks only (cheap): DBNET_EINVAL for malformed arguments, DBNET_ERANGE
 * when the request could never fit the pool.  Problems found on the device
 * at admission (bad edges, a delay over max_delay) fail that request alone:
 * state FAILED with the status code.  *id receives the request id (>= 1). */
int dbsrv_submit(dbsrv_t* s, const dbnet_graph_t* graph, const dbnet_region_params_t* params,
                 const dbsrv_request_t* request, int64_t* id);

/* One scheduling round: note the rounds the device has finished, copy the
 * results of requests that have run their steps, return cooled slots to the
 * pool, admit queued requests that fit (their graphs are copied on a second
 * stream while the device keeps stepping), and enqueue chunk_steps steps of
 * every resident request.  Blocks only when max_inflight rounds are already
 * enqueued, until the oldest finishes.  out may be NULL. */
int dbsrv_pump(dbsrv_t* s, dbsrv_stats_t* out);

/* Pump until no request is queued, running or cooling down. */
int dbsrv_drain(dbsrv_t* s);

int dbsrv_poll(dbsrv_t* s, int64_t id, dbsrv_status_t* out);

/* Results of a DONE request: BOLD samples [n][R] (as dbnet_read_bold) and
 * recorded spikes sorted by (step, id) (as dbnet_read_spikes).
 * DBNET_ESTATE when the request is not DONE, DBNET_ERANGE when cap is short. */
int dbsrv_read_bold(dbsrv_t* s, int64_t id, double* y, int64_t cap_samples, int64_t* n_out);
int dbsrv_read_spikes(dbsrv_t* s, int64_t id, int32_t* step, int32_t* nid, int64_t cap,
                      int64_t* n_out);

/* Forget a DONE or FAILED request, or cancel a QUEUED one (DBNET_ESTATE for
 * a running request). */
int dbsrv_release(dbsrv_t* s, int64_t id);

int dbsrv_stats(dbsrv_t* s, dbsrv_stats_t* out);

/* Waits for the device, then frees everything. */
void dbsrv_destroy(dbsrv_t* s);

#ifdef __cplusplus
}
#endif

#endif /* DBNET_H */

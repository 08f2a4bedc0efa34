/*
 * wmc.h -- C ABI of libwmc, the GB300 (sm_103a) hot path of the signed-particle
 * Wigner Monte Carlo method with the analytically weighted network kernel
 * (Sellier, Leygonie, Marceau Caron, arXiv:1806.00082).
 *
 * Plain C: every pointer argument is either a DEVICE pointer (marked [dev]) or
 * a HOST pointer (marked [host]); sizes are in elements unless stated.  The
 * caller allocates every buffer and keeps ownership; the library allocates no
 * device memory on any call below.  Every call is asynchronous on the given
 * stream unless it says it synchronises.  Argument errors are returned at once;
 * conditions found on the device (population too large, gamma dt >= 1, a
 * bounded wait that gave up) set flags in the workspace that wmc_get_error()
 * turns into a status and wmc_get_counters() reports.
 *
 * Notation (Sec. 2 of the paper):
 *   cells i = 0 .. n_x-1 of width dx, centre (i + 1/2) dx;
 *   coherence length L_C = Q dx (Q even), h = Q / 2;
 *   momentum index M in [-n_M/2, n_M/2), momentum M dp with dp = pi hbar / L_C;
 *   column k = M + n_M/2 of every [.. x n_M] array.
 *
 * Wigner kernel, Eq. (wigner-1d-discrete), with the network weight
 * w_l = -2 dx / (hbar L_C) of Sec. 2.2:
 *   V_W(i; M) = -(2 / (hbar Q)) sum_{m=1}^{h-1} sin(2 pi (m M mod Q) / Q) [V(i+m) - V(i-m)]
 * in 1/s for V in eV.  It is periodic in M with period Q, odd in M, and zero
 * at M = 0 and M = h, so a row is stored as its half period
 *   VWh[row][r] = V_W(i; r), r = 0 .. h-1  (VWh[row][0] = 0),
 * and V_W(i; M) = VWh[r], -VWh[Q - r] or 0 for r = M mod Q below, above or at h.
 *
 * Ensemble: the state is the net signed histogram hist[i][k] (int32,
 * row-major [n_x][n_M]) left by annihilation (rule 2: opposite signs in one
 * (cell, M) cancel).  Its survivors are numbered row-major over (i, k); the
 * particle with number id sits in cell i at a uniform offset f in [0, 1) drawn
 * at step t-1, the step that rebuilt it (see Random numbers below).
 * Step t (postulate, Sec. 2.1): every particle drifts, f' = fl32(f + D[M]) with
 * D[M] = fl32(M hbar pi dt / (m Q dx^2)) cells, and moves to the next or
 * previous cell when f' >= 1 or f' < 0 (leaving [0, n_x) absorbs it); in its new
 * cell c it creates a pair with probability gamma(c) dt, gamma = sum_M V_W^+
 * (Eq. momentum_integral), drawn as w 2^-32 < gamma dt; the pair sits in c with
 * signs +s, -s and momenta M + M', M - M', M' drawn from V_W^+(c; .) / gamma(c)
 * through the fixed-point CDF of wmc_kernel_cdf; children outside the momentum
 * grid are dropped (or wrapped).  Counts of parents and children in each
 * (cell, M) are summed with their signs: that sum is the annihilated state of
 * step t.
 * Calls and the method's objects: the particles of the postulate are the
 * histogram's survivors (wmc_materialize lists them: cell, offset, momentum,
 * sign); the kernel of the occupied cells is wmc_kernel_eval (rows) with
 * wmc_kernel_cdf (their CDF and gamma), or both at once into the workspace
 * with wmc_kernel_eval_occupied; wmc_annihilate enumerates the survivors and
 * the occupied cells, wmc_step advances them one step, wmc_density sums them
 * per cell, wmc_run chains the whole step.
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key (seed_lo, seed_hi).
 * Particle id takes word id % 4 of counter (id / 4, step, purpose, sim): the
 * offset with purpose REPOS = 2, u24(w) = (w >> 8) 2^-24, at the step that
 * rebuilt it; the pair-creation word with purpose GEN = 1 at step t.  A created
 * pair draws U2 = (w0 >> 5) 2^26 + (w1 >> 6) from counter (id, t, PICK = 3, sim).
 */
#ifndef WMC_H_
#define WMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* wmc_stream_t;

typedef struct wmc_params {
  double dx_m;          /* cell width dx [m] */
  double mass_kg;       /* particle mass [kg] */
  double dt_s;          /* time step [s] */
  uint64_t seed;        /* Philox key (low word, high word) */
  int32_t n_x;          /* cells, 1 .. 2^24 */
  int32_t Q;            /* quadrature points L_C / dx, even, 2 .. 4096 */
  int32_t n_M;          /* momentum indices, even, 2 .. 4096 */
  int32_t bc_potential; /* 0: V = 0 outside [0, n_x); 1: V takes the edge value */
  int32_t child_wrap;   /* 0: drop children outside the momentum grid; 1: wrap */
  uint32_t sim;         /* simulation index: Philox counter word 3 */
} wmc_params;

typedef enum wmc_status {
  WMC_OK = 0,
  WMC_ERR_ARG = 1,          /* bad argument or parameter */
  WMC_ERR_CAPACITY = 2,     /* population >= 2^32 or output capacity too small */
  WMC_ERR_RATE = 3,         /* gamma dt >= 1 in an evaluated cell */
  WMC_ERR_CUDA = 4,         /* a CUDA runtime call failed */
  WMC_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  WMC_ERR_UNSUPPORTED = 6   /* precision or shape not supported by this build */
} wmc_status;

/* Input precision of the sine x dV contraction (accumulation is FP32).
 * WMC_FP32 asks for FP32 accuracy and lets the library choose the form: the
 * 3xTF32 tensor-core form for windows Q > 256 (its split kernel keeps the
 * TF32 hi x hi product of every K block in its own accumulator and sums the
 * blocks in FP32 registers; measured normwise error 3.6e-7 at Q = 1024 and
 * 4.9e-7 at Q = 2048 against 2.9e-7 for the CUDA-core form, at 3x its speed),
 * and in wmc_kernel_eval / wmc_kernel_eval_rows also for 128 <= Q <= 256 when
 * the rows number at least 128 per SM; the CUDA-core form otherwise (smaller
 * windows and row counts, the step loop's fused small-window stage, the N = 2
 * network, windows the split kernel does not hold).  WMC_FP32_SIMT always
 * takes the CUDA-core form.  The FP16 split is faster still but FP16's exponent range (|dV| below
 * 65504 eV, full precision for |dV| above about 1e-4 eV) makes its accuracy
 * depend on the potential's scale, so it stays an explicit choice. */
typedef enum wmc_precision {
  WMC_FP32 = 0,        /* FP32 accuracy, form chosen by the library (above) */
  WMC_BF16 = 1,        /* BF16 inputs on the tensor cores */
  WMC_FP16 = 2,        /* FP16 inputs on the tensor cores */
  WMC_FP16_SPLIT = 3,  /* FP16 hi/lo split, three tensor-core products */
  WMC_TF32X3 = 4,      /* TF32 hi/lo split, three tensor-core products */
  WMC_FP32_SIMT = 5    /* FP32 inputs, compensated FP32 accumulation on the CUDA cores */
} wmc_precision;

/* Device flags, readable with wmc_get_counters(). */
#define WMC_FLAG_RATE 1u      /* an evaluated cell had gamma dt >= 1 (events then always fire) */
#define WMC_FLAG_CAPACITY 2u  /* population >= 2^32 (the step did nothing) or a capacity was short */
#define WMC_FLAG_TIMEOUT 4u   /* a bounded device wait gave up */

/* Counters kept in the workspace, cumulative since wmc_init / wmc_reset_counters. */
typedef struct wmc_counters {
  uint64_t population;      /* survivors enumerated by the last wmc_annihilate */
  uint64_t particle_steps;  /* sum over steps of the population at step start */
  uint64_t pairs;           /* pairs created */
  uint64_t absorbed;        /* particles that left [0, n_x) */
  int64_t absorbed_signed;  /* sum of their signs */
  uint64_t dropped;         /* children outside the momentum grid (drop mode) */
  int64_t dropped_signed;   /* sum of their signs */
  int32_t n_occ;            /* cells whose kernel the last step evaluated */
  int32_t n_items;          /* work items of the last step */
  uint32_t flags;           /* WMC_FLAG_* */
  uint32_t step;            /* device step counter used by wmc_run */
} wmc_counters;

/* Library version string. */
const char* wmc_version(void);

/* Static description of a status code. */
const char* wmc_status_string(wmc_status s);

/* Bytes of device workspace for these parameters (0 if they are invalid).
 * The workspace holds the survivor enumeration, the occupied-cell list, the
 * kernel rows, CDFs and thresholds of up to n_x cells, the drift table, the
 * sine matrices and the counters.  Allocate it once per simulation, aligned
 * to 256 bytes (any cudaMalloc / torch allocation is). */
size_t wmc_workspace_size(const wmc_params* p);

/* Checks p, fills the workspace's constant tables (drift D, sine matrices)
 * and zeroes its counters.  ws [dev] of ws_bytes >= wmc_workspace_size(p).
 * Must precede every other call that takes ws.  Stream-ordered. */
wmc_status wmc_init(const wmc_params* p, void* ws, size_t ws_bytes, wmc_stream_t stream);

/* Zeroes the counters and flags of an initialised workspace. */
wmc_status wmc_reset_counters(const wmc_params* p, void* ws, wmc_stream_t stream);

/* Numbering of a sub-domain's particles (domain decomposition over cell
 * ranges): the survivors enumerated by wmc_annihilate and the steps of wmc_run
 * are numbered from id_base (0 after wmc_init) instead of 0, so a rank that
 * owns a range of cells, its histogram zero outside the range, draws the
 * Philox words of the global numbering when id_base is the number of
 * particles in the cells before its range.  Particles that drift out of the
 * range land in the neighbouring rows of the output, for the owning rank to
 * add.  id_base + the population must stay below 2^32 (else WMC_FLAG_CAPACITY);
 * wmc_materialize writes survivor id at place id - id_base.  Stream-ordered;
 * WMC_ERR_ARG for id_base >= 2^32. */
wmc_status wmc_set_id_base(const wmc_params* p, void* ws, uint64_t id_base, wmc_stream_t stream);

/* Failure-detection check of the device wait pattern the tensor-core kernels
 * use: one device thread waits until the 32-bit word *signal [dev] is non-zero
 * or max_cycles SM clock cycles have passed; if it gives up it sets
 * WMC_FLAG_TIMEOUT in the workspace flags (read with wmc_get_counters, cleared
 * by wmc_reset_counters) and returns, so the context stays usable.  The
 * library writes nothing else; max_cycles 0 .. 2^34 (about eight seconds).
 * Stream-ordered. */
wmc_status wmc_check_wait(const wmc_params* p, const uint32_t* signal, uint64_t max_cycles, void* ws,
                          wmc_stream_t stream);

/* Timing of the particle-step kernel (a measurement aid; the paper has no
 * counterpart).  While enable != 0, every wmc_step and every step of wmc_run
 * records two CUDA events owned by the library on the launching stream, right
 * before and right after the particle-step kernel (one pair per device, for
 * devices 0-7; steps on other devices are not timed; when
 * the stream is being captured they become event-record nodes, and the cached
 * step graphs are recaptured whenever the setting changes).  The events add
 * latency to a step graph (a few microseconds per event node) but no work,
 * and change none of its results.  Host call; always WMC_OK. */
wmc_status wmc_step_timing(int32_t enable);

/* Waits for the most recently recorded pair of the current device and writes
 * the milliseconds between them to *ms [host]: the duration of the last
 * particle-step kernel that ran with timing on (of a step-pair graph, the
 * second step's).  WMC_ERR_ARG for a null ms, WMC_ERR_UNSUPPORTED if no pair
 * has been recorded on this device, WMC_ERR_CUDA on a CUDA error. */
wmc_status wmc_step_timing_read(float* ms);

/* Reads the counters (synchronises the stream).  out [host]. */
wmc_status wmc_get_counters(const wmc_params* p, const void* ws, wmc_counters* out, wmc_stream_t stream);

/* The device conditions of the workspace as a status: synchronises the stream,
 * reads the flags and writes to *device_status [host] WMC_ERR_TIMEOUT,
 * WMC_ERR_CAPACITY or WMC_ERR_RATE (in that order of precedence) if the
 * corresponding flag is set, else WMC_OK, and a NUL-terminated description
 * into msg [host] of len bytes (may be NULL).  The flags stay set until
 * wmc_reset_counters.  Returns WMC_ERR_ARG for bad arguments, WMC_ERR_CUDA if
 * the read fails. */
wmc_status wmc_get_error(const wmc_params* p, const void* ws, wmc_stream_t stream, wmc_status* device_status,
                         char* msg, size_t len);

/* ---------------------------------------------------------------------------
 * Kernel evaluation on given cells -- Eq. (wigner-1d-discrete) as the N = 1
 * analytic network of Sec. 2.2 (hidden units V(l) sin(theta_l), output weight
 * w_l): a contraction of the potential differences against the integer-indexed
 * sine matrix S[m][r] = sin(2 pi (m r mod Q) / Q).
 *   V    [dev] float[n_x], eV.
 *   occ  [dev] int32[n_occ], cells in [0, n_x) (any order, repeats allowed).
 *   n_occ 0 .. n_x (host value).
 *   prec WMC_FP32 (FP32 accuracy, form chosen as described at wmc_precision),
 *        WMC_FP32_SIMT or a tensor-core form (WMC_ERR_UNSUPPORTED if not built).
 *   VWh  [dev] float[n_occ][Q/2], half-period rows (layout above); written.
 * ------------------------------------------------------------------------- */
wmc_status wmc_kernel_eval(const wmc_params* p, const float* V, const int32_t* occ, int32_t n_occ,
                           wmc_precision prec, float* VWh, void* ws, wmc_stream_t stream);

/* Same evaluation as wmc_kernel_eval for callers that cannot allocate device
 * memory or pass a workspace (the paper has no counterpart: this serves
 * embedding).  Such callers are, for example, code inside an application whose
 * device memory belongs to a pool allocator (a cudaMalloc there may fail,
 * stall, synchronise the device or go unaccounted), or applications that
 * allocate everything at start-up and forbid it afterwards.  The only scratch
 * of the evaluation, the sine matrix, lives in a fixed 1 MiB array in the
 * library's device memory, which every GPU that loads the library holds until
 * the process exits; no call allocates.
 *   Limit: Q <= 1024, else WMC_ERR_CAPACITY (nothing is launched).
 *   V, occ, n_occ, VWh as for wmc_kernel_eval with WMC_FP32_SIMT (the same
 *   tiled CUDA-core kernel and sine values: bit-identical for Q > 256).
 *   Every call looks up the array's device address in the current context
 *   (no address outlives a context, e.g. across cudaDeviceReset); make the
 *   first call of a process before any stream capture, since it may load the
 *   library's device code.  All calls share the array and each refills what it reads, so
 *   calls that overlap on the GPU (other streams, other threads) race on it:
 *   serialise them. */
wmc_status wmc_kernel_eval_noalloc(const wmc_params* p, const float* V, const int32_t* occ, int32_t n_occ,
                                   float* VWh, wmc_stream_t stream);

/* Eq. (wigner-1d-discrete) on every cell by a sliding window, in FP64: for
 * each half-period column r, W(i) = sum_{l=i-h}^{i+h} V(l) exp(i 2 pi l r / Q)
 * moves by one term in and one out per cell and VWh[i][r] =
 * -(2 / (hbar Q)) Im[exp(-i 2 pi i r / Q) W(i)], so all n_x rows cost O(n_x h)
 * FP64 operations (the window sum started afresh every 256 cells) instead of
 * O(n_x h^2); exact integer phases.  An independent arrangement of the sum,
 * accurate to the FP32 rounding of the output, for cross-checking the other
 * forms on every cell.  V [dev] float[n_x] in eV; VWh [dev] float[n_x][Q/2]
 * (row = cell), written; ws as for wmc_kernel_eval (its 2Q-double phase table
 * is overwritten). */
wmc_status wmc_kernel_eval_dft(const wmc_params* p, const float* V, float* VWh, void* ws, wmc_stream_t stream);

/* The N = 2 network of Sec. 2.3 -- Eq. (kernel_ML) with N = 2 and the
 * barycentric weights (omega^V = (1, 1), omega^theta = (1/2, 1/2),
 * W_l = w_l = -2 dx / (hbar L_C), one cosine factor): the terms V(l) sin(theta_l)
 * of the N = 1 network are grouped by consecutive cells (2q, 2q + 1), the
 * potential of a pair replaced by its average, so that
 *   V_W2(i; M) = -(2 / (hbar Q)) cos(pi M / Q)
 *                sum_{pairs (2q, 2q+1) in [i - h, i + h]} [V(2q) + V(2q+1)] sin(pi (4q + 1 - 2i) M / Q),
 * half as many sines as the N = 1 network's 2h + 1 terms.  It is odd and
 * Q-periodic in M and zero at M = 0 and M = h, so rows use the same
 * half-period layout; it equals wmc_kernel_eval where V is constant on every
 * pair of cells and approaches it to first order in dx for a smooth V.
 * Evaluated as a contraction of the signed pair sums A(i, u) (u = 0 .. h - 1:
 * V(i+u) + V(i+u+1) if i + u is even, else -(V(i-u-1) + V(i-u))) with
 * cos(pi r / Q) sin(pi (2u + 1) r / Q).
 *   V, occ, n_occ, VWh, ws as for wmc_kernel_eval.
 *   prec WMC_FP32, WMC_BF16, WMC_FP16 or WMC_FP16_SPLIT (WMC_TF32X3 and
 *        windows whose operands do not fit return WMC_ERR_UNSUPPORTED).
 * The rows can drive the simulation through wmc_kernel_table_occupied. */
wmc_status wmc_kernel_eval_n2(const wmc_params* p, const float* V, const int32_t* occ, int32_t n_occ,
                              wmc_precision prec, float* VWh, void* ws, wmc_stream_t stream);

/* The trained N = 2 network of Sec. 2.3: Eq. (kernel_ML) with N = 2 whose
 * weights are learnt by stochastic gradient descent on a mean-squared-error
 * loss against exact kernels.  Reduced units (kernels times hbar Q / 2, V in eV):
 *   y(i, j) = cos(pi j / Q) sum_{d in D(i)} W[d] (wv1 V(i + d) + wv2 V(i + d + 1))
 *                                           sin(2 pi j / Q (wt1 d + wt2 (d + 1))),
 * D(i) = {d in [-h, h - 1] : i + d even} (the absolute pairs (2q, 2q + 1)
 * inside the window), W indexed by d + h.  A parameter vector is
 * float[Q + 4] = [W[0 .. Q-1], wv1, wv2, wt1, wt2]; W = -1, wv = (1, 1),
 * wt = (1/2, 1/2) is the analytic N = 2 network (wmc_kernel_eval_n2).
 * Loss of an example: mean over cells i and columns j = 1 .. h - 1 of
 * (y - t)^2; one SGD step per example, p <- p - lr dL/dp.
 *   V      [dev] float[n_examples][n_x] potentials (eV).
 *   VW     [dev] float[n_examples][n_x][Q/2] their exact kernels in 1/s, half
 *          period (columns j = 0 .. h - 1, e.g. from wmc_kernel_eval_rows).
 *   order  [dev] int32[epochs][n_examples]: the examples of each epoch in turn.
 *   lr     [dev] float[n_runs]: runs train the same examples in the same order,
 *          one learning rate each (one thread block per run).
 *   params [dev] float[n_runs][Q + 4]: initial weights in, trained weights out.
 *   loss   [dev] float[n_runs][epochs] or NULL: mean loss of each epoch (each
 *          step's loss taken before its update).
 * n_x even; WMC_ERR_UNSUPPORTED if n_x (Q/2 + 1) + Q^2 floats exceed the shared
 * memory of one block (about 200 KB).  Deterministic for given inputs. */
wmc_status wmc_n2_train(const wmc_params* p, int32_t n_examples, const float* V, const float* VW, int32_t epochs,
                        const int32_t* order, int32_t n_runs, const float* lr, float* params, float* loss,
                        wmc_stream_t stream);

/* Rows of the trained N = 2 network in 1/s for parameters params [dev]
 * float[Q + 4] (layout as wmc_n2_train): V [dev] float[n_pot][n_x];
 * VWh [dev] float[n_pot n_x][Q/2], row b n_x + i = cell i of potential b, half
 * period.  The rows can drive the simulation through wmc_kernel_table_occupied. */
wmc_status wmc_n2_eval(const wmc_params* p, const float* params, const float* V, int32_t n_pot, float* VWh,
                       wmc_stream_t stream);

/* gamma and the momentum CDF of kernel rows -- Eq. (momentum_integral) and the
 * postulate's draw of p' with probability V_W^+ / gamma.  The positive parts
 * x_k = max(V_W(k), 0) of a row are quantised relative to the row maximum:
 *   e = floor(log2 max_k x_k),  s = 61 - ceil(log2 n_M) - e,
 *   q_k = x_k 2^s rounded to the nearest integer (ties to even),
 * so that the CDF is the exact integer running sum
 *   cdf[row][k] = sum_{k' <= k} q_k'  (< 2^62)
 * and gamma[row] = fl64(cdf[row][n_M - 1] 2^-s) (resolution 2^-52 of the row
 * maximum, like an FP64 sum, but exact and independent of summation order).
 * p' takes the smallest k with cdf[k] > floor(U2 cdf[n_M-1] / 2^53) for a
 * 53-bit uniform integer U2.  A row without positive entries has gamma = 0.
 *   VWh   [dev] float[n_rows][Q/2].
 *   cdf   [dev] int64[n_rows][n_M] (row-major) or NULL.
 *   gamma [dev] double[n_rows].
 *   scale [dev] int32[n_rows] (receives s) or NULL. */
wmc_status wmc_kernel_cdf(const wmc_params* p, const float* VWh, int32_t n_rows, int64_t* cdf, double* gamma,
                          int32_t* scale, wmc_stream_t stream);

/* ---------------------------------------------------------------------------
 * The simulation step, as three stream-ordered calls on one workspace:
 *   wmc_annihilate(hist_t-1)  -> survivor enumeration + occupied cells
 *   wmc_kernel_eval_occupied  -> V_W, CDF, gamma on those cells
 *   wmc_step(hist_t-1 -> hist_t)
 * wmc_run() chains them for many steps (in a CUDA graph where it can).
 * ------------------------------------------------------------------------- */

/* Rule 2 rebuild: enumerates the survivors of the net histogram hist [dev]
 * int32[n_x][n_M] (row-major ids, work items of 512 to 2048 ids of one cell, sized from the previous population), marks the
 * cells the next drift can reach (occupied cells and their neighbour in each
 * drift direction present) as the occupied list for the kernel, and, if
 * rho [dev] int64[n_x] is not NULL, writes the density (rule 1) of hist.
 * A population >= 2^32 sets WMC_FLAG_CAPACITY and the next step does nothing. */
wmc_status wmc_annihilate(const wmc_params* p, const int32_t* hist, int64_t* rho, void* ws,
                          wmc_stream_t stream);

/* Kernel rows, CDFs and event thresholds for the occupied list of the last
 * wmc_annihilate, kept in the workspace.  V [dev] float[n_x] in eV. */
wmc_status wmc_kernel_eval_occupied(const wmc_params* p, const float* V, wmc_precision prec, void* ws,
                                    wmc_stream_t stream);

/* Same, but the kernel values come from a caller table instead of the
 * contraction (e.g. a trained network's output): table [dev] float[n_x][Q/2]
 * half-period rows for every cell. */
wmc_status wmc_kernel_table_occupied(const wmc_params* p, const float* table, void* ws,
                                     wmc_stream_t stream);

/* Step t >= 1 of the postulate (drift, absorption, pair creation, histogram of
 * parents and children): reads hist_in [dev] (the state left by step t-1, as
 * enumerated by the last wmc_annihilate) and writes the net histogram of step
 * t to hist_out [dev] int32[n_x][n_M] (overwritten; must not alias hist_in). */
wmc_status wmc_step(const wmc_params* p, const int32_t* hist_in, uint32_t t, int32_t* hist_out, void* ws,
                    wmc_stream_t stream);

/* n_steps steps t = t_first .. t_first + n_steps - 1 starting from hist_a [dev]
 * (the state after step t_first - 1), using hist_b [dev] as the second
 * buffer; the final state is left in hist_a.  prec selects the kernel form.
 * use_graph != 0 captures the step pair, and for an odd n_steps the last step
 * with its copy back to hist_a, in cached CUDA graphs (not on the legacy
 * default stream, where it runs the calls directly); the graphs of the last
 * four configurations (parameters, buffers, workspace, precision, stream) are
 * kept, so alternating between buffer sets does not recapture. */
wmc_status wmc_run(const wmc_params* p, const float* V, int32_t* hist_a, int32_t* hist_b, uint32_t t_first,
                   int32_t n_steps, wmc_precision prec, int32_t use_graph, void* ws, wmc_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched form: n_sims independent simulations of uneven size (each with its
 * own wmc_params, potential, net histogram and Philox stream, counter word 3 =
 * its sim field) advanced together, one launch per phase for the whole batch.
 * Each simulation's result is bit-identical to running it alone.  Supported
 * for the FP32 kernel and Q <= 256.  Concatenated buffers: the potentials
 * V [dev] float[sum n_x] and histograms [dev] int32[sum n_x n_M], simulation s
 * at the offsets wmc_batch_layout returns.
 * ------------------------------------------------------------------------- */

/* Bytes of batch workspace (0 if any parameter set is invalid or Q > 256). */
size_t wmc_batch_workspace_size(const wmc_params* ps, int32_t n_sims);

/* Offsets of simulation s in the concatenated potentials (cell_off[s]) and
 * histograms (hist_off[s]); both [host] int64[n_sims + 1], the last entry is
 * the total. */
wmc_status wmc_batch_layout(const wmc_params* ps, int32_t n_sims, int64_t* cell_off, int64_t* hist_off);

/* Fills the batch workspace (descriptors, tables, counters).  Synchronises the
 * stream once (it copies the per-simulation descriptors from the host). */
wmc_status wmc_batch_init(const wmc_params* ps, int32_t n_sims, void* ws, size_t ws_bytes, wmc_stream_t stream);

/* n_steps steps of every simulation from hist_a (state after step
 * t_first - 1), hist_b the second buffer, final state in hist_a.
 * per_thread: survivor ids per lane of a work item (4, 8, 16, 32, 64, 128 or
 * 256; 0 = 16), e.g. from wmc_batch_autotune; results do not depend on it.  use_graph
 * as for wmc_run. */
wmc_status wmc_batch_run(const wmc_params* ps, int32_t n_sims, const float* V, int32_t* hist_a, int32_t* hist_b,
                         uint32_t t_first, int32_t n_steps, int32_t per_thread, int32_t use_graph, void* ws,
                         wmc_stream_t stream);

/* Times one batch step from hist (left unchanged; scratch [dev] receives the
 * output) for each candidate work-item size and writes the fastest to
 * *best_per_thread [host].  Synchronises. */
wmc_status wmc_batch_autotune(const wmc_params* ps, int32_t n_sims, const float* V, int32_t* hist, int32_t* scratch,
                              uint32_t t, void* ws, int32_t* best_per_thread, wmc_stream_t stream);

/* Counters of the batch (totals over all simulations); synchronises. */
wmc_status wmc_batch_get_counters(const wmc_params* ps, int32_t n_sims, const void* ws, wmc_counters* out,
                                  wmc_stream_t stream);

/* ---------------------------------------------------------------------------
 * Differentiation form: the kernel rows and gamma as functions of a smooth
 * potential, and their adjoint.
 *   V(x) = sum_b h_b T(x; c_b - w_b/2, c_b + w_b/2) + sum_s o_s T(x; s L/ns, (s+1) L/ns),
 *   T(x; a, b) = (tanh((x - a)/eps) - tanh((x - b)/eps)) / 2,  x = (i + 1/2) dx,
 * lengths in nm, energies in eV; theta [dev] float[n_pot][3 nb + ns] per
 * potential = [h_0..h_{nb-1}, w_0.., c_0.., o_0..o_{ns-1}].
 * ------------------------------------------------------------------------- */

/* V [dev] float[n_pot][n_x] from theta. */
wmc_status wmc_potential_tanh(const wmc_params* p, const float* theta, int32_t n_pot, int32_t n_barriers,
                              int32_t n_segments, float eps_nm, float* V, wmc_stream_t stream);

/* theta_bar [dev] float[n_pot][3 nb + ns] = sum_i Vbar[i] dV(x_i)/d theta. */
wmc_status wmc_potential_tanh_vjp(const wmc_params* p, const float* theta, int32_t n_pot, int32_t n_barriers,
                                  int32_t n_segments, float eps_nm, const float* Vbar, float* theta_bar,
                                  wmc_stream_t stream);

/* Kernel rows of every cell of n_pot potentials V [dev] float[n_pot][n_x]:
 * VWh [dev] float[n_pot * n_x][Q/2] (row b n_x + i = cell i of potential b);
 * gamma follows from wmc_kernel_cdf on these rows.  Any precision form. */
wmc_status wmc_kernel_eval_rows(const wmc_params* p, const float* V, int32_t n_pot, wmc_precision prec, float* VWh,
                                void* ws, wmc_stream_t stream);

/* Adjoint of wmc_kernel_eval_rows and of gamma (Eq. wigner-1d-discrete and
 * Eq. momentum_integral): for upstream gradients gVW [dev] float[rows][Q/2]
 * and g_gamma [dev] float[rows] (either may be NULL; rows = n_pot n_x) of the
 * rows VWh, writes Vbar [dev] float[n_pot][n_x] = dL/dV.
 *   Gbar = gVW + g_gamma (cnt_pos(r) [VWh > 0] - cnt_neg(r) [VWh < 0]),
 *   Abar[i][m] = c sum_r Gbar[i][r] S[m][r],  Vbar[l] = sum_m Abar[l-m][m] - Abar[l+m][m],
 * cnt_pos(r) / cnt_neg(r) = momentum indices M of the grid with M = r / M = -r (mod Q).
 * Abar [dev] float[rows][Q/2] is caller scratch.  bc_potential 0 and Q <= 256.
 * The Abar contraction runs on the tensor cores as 3xTF32 (TF32 hi/lo parts
 * of Gbar and of S, per-K-block accumulators: FP32-level accuracy at the FP32
 * exponent range of the gradients); the scatter to Vbar on the CUDA cores. */
wmc_status wmc_kernel_vjp(const wmc_params* p, const float* VWh, const float* gVW, const float* g_gamma,
                          int32_t n_pot, float* Abar, float* Vbar, void* ws, wmc_stream_t stream);

/* Rule 1: rho[i] = sum_k hist[i][k].  hist [dev] int32[n_x][n_M], rho [dev] int64[n_x]. */
wmc_status wmc_density(const wmc_params* p, const int32_t* hist, int64_t* rho, wmc_stream_t stream);

/* Explicit survivors of the last wmc_annihilate, as rebuilt at step t (the
 * offset of id is u24 of word id % 4 of Philox(id / 4, t, REPOS, sim)): SoA arrays [dev] of
 * capacity elements, written in id order.  If the population exceeds capacity
 * nothing is written and WMC_FLAG_CAPACITY is set. */
wmc_status wmc_materialize(const wmc_params* p, const int32_t* hist, uint32_t t, int32_t* cell, float* f,
                           int16_t* M, int8_t* sign, int64_t capacity, void* ws, wmc_stream_t stream);

/* Philox4x32-10 of n counters ctr [dev] uint32[n][4] under key (key0, key1),
 * out [dev] uint32[n][4].  The generator the step uses, exposed for checks. */
wmc_status wmc_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, int64_t n, uint32_t* out,
                             wmc_stream_t stream);

/* Throughput probe of the generator (a measurement aid; the paper has no
 * counterpart): n_threads threads (a multiple of 256) each evaluate
 * 2 pairs_per_thread Philox4x32-10 calls, two at a time under one key
 * schedule as the particle step does, on distinct counters (pairs_per_thread
 * n_threads < 2^32), and write the XOR of all their words to out [dev]
 * uint32[n_threads].  Timing it with events gives the calls per second the
 * GPU sustains on the generator alone, the ceiling of the particle step's
 * arithmetic.  Stream-ordered. */
wmc_status wmc_philox_throughput(uint32_t key0, uint32_t key1, int32_t pairs_per_thread, uint32_t* out,
                                 int64_t n_threads, wmc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* WMC_H_ */

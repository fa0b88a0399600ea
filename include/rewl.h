/*
 * rewl.h -- C ABI of the GB300 replica-exchange Wang-Landau (REWL) library.
 *
 * Method: T. Vogel, Y. W. Li, T. Wuest, D. P. Landau, "Scalable replica-exchange
 * framework for Wang-Landau sampling", arXiv:1407.5140.
 *
 * The library samples the density of states g(E) of the 2D Ising model and the
 * 2D q-state Potts model (Sec. III A, Eq. (2)) on L x L periodic lattices (J = 1)
 * with h overlapping energy windows and m independent Wang-Landau walkers per
 * window (Sec. II A, Fig. 1); walkers of neighbouring windows swap
 * configurations with the probability of Eq. (1), alternating between the two
 * sets of window pairs (Fig. 2); walkers of one window average their ln g after
 * each Wang-Landau iteration (Sec. II A).  All compute runs in the library's
 * sm_103a CUDA kernels; there is no CPU fallback.
 *
 * Conventions
 *  - Energies are integers in units of J.  Ising: E = -sum s_i s_j, bins of 4
 *    (E = -2N + 4b).  Potts: E = -sum delta(q_i, q_j), bins of 1 (E = -2N + b).
 *    The caller names an inclusive energy range [e_min, e_max] (Sec. II A,
 *    "between E_min and E_max"); bins are numbered from e_min.
 *  - ln g is held on the device as signed 64-bit fixed point in units of 2^-32.
 *    Every value the method produces (sums of ln f = 2^-k and means rounded to
 *    2^-32) is exactly representable, and converts exactly to FP64 while
 *    |ln g| < 2^21; the library reports REWL_EDEVICE if a value leaves that range.
 *  - Every entry point returns a rewl_status; none throws or aborts.  After a
 *    device error the context is sticky-failed (REWL_ESTATE) and
 *    rewl_last_error() describes the first failure.
 *  - Results are a pure function of the instance descriptors and seeds: they do
 *    not depend on batching, on launch configuration or on the autotuner.
 *  - The library owns all device memory it allocates in rewl_create*(); host
 *    buffers passed in are owned by the caller and only read or written during
 *    the call (the library synchronises its stream before touching them).
 *  - Work is enqueued on the stream given at creation (NULL: a stream the
 *    library creates).  rewl_run / rewl_exchange return once the work is
 *    enqueued; read-out calls synchronise.
 *  - Distinct contexts may be driven from different host threads at the same
 *    time (each has its own device memory, streams and CUDA graph, captured
 *    in thread-local mode); one context must not be used by two threads at
 *    once.
 */
#ifndef REWL_H
#define REWL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rewl_ctx rewl_ctx;

typedef enum {
    REWL_OK = 0,
    REWL_EINVAL = -1,    /* an argument is out of range (message says which) */
    REWL_ENOMEM = -2,    /* device or host allocation failed                 */
    REWL_ECUDA = -3,     /* a CUDA runtime call failed                       */
    REWL_ETIMEOUT = -4,  /* a bounded device wait gave up                    */
    REWL_ESTATE = -5,    /* context already failed, or call out of order     */
    REWL_EDEVICE = -6    /* a kernel raised its error word                   */
} rewl_status;

typedef enum { REWL_ISING = 0, REWL_POTTS = 1 } rewl_model;

/* One independent REWL problem (Sec. II A notation: h windows, m walkers per
 * window, overlap o with the next-lower window). */
typedef struct rewl_instance {
    int32_t model;              /* rewl_model                                   */
    int32_t L;                  /* even, 4 <= L <= 512                          */
    int32_t q;                  /* Potts states, 2..127 (ignored for Ising)     */
    int32_t n_windows;          /* h >= 1                                       */
    int64_t e_min, e_max;       /* inclusive energy range, on the bin grid      */
    double overlap;             /* o in [0, 1)                                  */
    int32_t walkers_per_window; /* m, 1..32                                     */
    int32_t flat_rule;          /* 0: flat iff min H >= p <H> (Sec. II A);
                                 * 1: Zhou-Bhatt, flat iff min H >= a/sqrt(ln f)
                                 *    (Sec. IV B, Eq. (8)), a = flatness; both
                                 *    over the window's realisable bins       */
    double flatness;            /* rule 0: p in (0, 1]; rule 1: a in (0, 1e6]  */
    double ln_f_final;          /* run ends after the stage with ln f <= this   */
    uint64_t seed;              /* Philox key                                   */
    uint32_t instance_id;       /* xor-ed into the key's high word              */
    uint32_t reserved2;
} rewl_instance;

/* Create one instance (a batch of one).  Allocates the device state, builds the
 * windows of Sec. II A / Fig. 1 (equal widths w = ceil(B / (1 + (h-1)(1-o))),
 * lo_i = floor(i (B - w) / (h - 1))) and brings every walker into its window
 * (init kernel).  cuda_stream: a cudaStream_t, or NULL. */
rewl_status rewl_create(rewl_ctx **out, rewl_model model, int L, int q,
                        long e_min, long e_max, int n_windows, double overlap,
                        int walkers_per_window, double flatness, double ln_f_final,
                        unsigned long long seed, void *cuda_stream);

/* Create n_inst independent instances of any mix of models and sizes, sampled
 * together by the same launches (persistent batch).  inst: host array, read
 * during the call. */
rewl_status rewl_create_batch(rewl_ctx **out, const rewl_instance *inst, int n_inst,
                              void *cuda_stream);

/* As rewl_create_batch, with every window given bin by bin instead of by the
 * equal-width rule: windows of different widths, e.g. sized so that they
 * finish their WL iterations at a similar pace (the run-time-balanced windows
 * of Sec. V).  lo, hi: host arrays of sum(inst[k].n_windows) bin indices,
 * instance after instance; window i of an instance covers bins lo[i]..hi[i]
 * (inclusive).  Per instance the windows must start at bin 0, end at bin
 * B - 1, have increasing lower and upper ends, overlap their neighbour by at
 * least one bin and be at least 2 * (largest bin change) + 1 bins wide (5
 * Ising, 9 Potts); otherwise REWL_EINVAL.  The instance's `overlap` field is
 * not used.  Read during the call. */
rewl_status rewl_create_batch_windows(rewl_ctx **out, const rewl_instance *inst, int n_inst,
                                      const int32_t *lo, const int32_t *hi, void *cuda_stream);

/* n_sweeps Wang-Landau sweeps of every walker (one sweep = N single-spin
 * trials, Sec. IV A), each trial accepted with min(1, g(E)/g(E')), followed by
 * ln g(E) += ln f and H(E) += 1 (Sec. II A).  After every `check_every` sweeps
 * (default 1) each walker's flatness is tested; when all m walkers of a window
 * are flat their ln g are averaged, H is reset and ln f halves, or the window
 * converges once ln f <= ln_f_final and then keeps walking (and exchanging)
 * with ln g frozen and H no longer counted. */
rewl_status rewl_run(rewl_ctx *ctx, long n_sweeps);

/* One replica-exchange phase (Eq. (1), Fig. 2): window pairs (i, i+1) with
 * i = t mod 2, t = number of earlier calls; walker j of window i proposes to
 * swap configurations with walker (j + s) mod m of window i+1. */
rewl_status rewl_exchange(rewl_ctx *ctx);

/* `n_cycles` times: rewl_run(sweeps_per_cycle) then rewl_exchange(), replayed
 * from one captured CUDA graph. */
rewl_status rewl_run_cycles(rewl_ctx *ctx, long n_cycles, long sweeps_per_cycle);

/* Alternate `exchange_interval` sweeps and one exchange phase until every
 * window of every instance has converged or max_sweeps were done; polls the
 * device every `poll_cycles` cycles.  *converged = 1 on success. */
rewl_status rewl_run_to_convergence(rewl_ctx *ctx, long exchange_interval, long max_sweeps,
                                    long poll_cycles, int *converged);

/* ln g of instance `inst`.  per_window = 1: the h pieces, h*w values, each the
 * walker mean of its window (identical after a merge; NaN past the end of a
 * window narrower than w).  per_window = 0: the
 * pieces joined as in Sec. II B (five-point inverse-temperature estimate,
 * join where the pieces' estimates agree best) and normalised so that
 * ln g(e_min) = ln 2 (Ising) or ln q (Potts); B values, NaN on energies no
 * configuration has.  e_of_bin (may be NULL) receives the energies.
 * *n_written: values written; REWL_EINVAL if cap is too small. */
rewl_status rewl_get_dos(rewl_ctx *ctx, int inst, double *ln_g, long cap, long *n_written,
                         long *e_of_bin, int per_window);

/* The joining of rewl_get_dos (Sec. II B) applied to pieces the caller
 * supplies, e.g. means of pieces over independent runs, or bootstrap
 * resamples of them (Sec. II B, last paragraph).  Host-only: needs no context
 * and no GPU.  h windows; pieces: h rows of w doubles, window i's bins
 * lo[i] .. lo[i] + ww[i] - 1 at the start of row i; reach: B flags (1 =
 * realisable energy); bin_width: energy per bin (4 Ising, 1 Potts); the result
 * (B doubles, NaN on unrealisable bins) is shifted so the first realisable bin
 * holds ln_g_first (ln 2 Ising, ln q Potts).  The windows must cover bins
 * 0 .. B - 1, overlap their neighbours with increasing ends and be at least 5
 * bins wide (REWL_EINVAL otherwise, message in rewl_last_error(NULL)). */
rewl_status rewl_join_pieces(int h, int w, int B, const int32_t *lo, const int32_t *ww,
                             const uint8_t *reach, double bin_width, double ln_g_first,
                             const double *pieces, double *ln_g);

/* Sweep count at which each window of instance `inst` ended each Wang-Landau
 * stage k = 0..32 (ln f = 2^-k) with the merge of its walkers' ln g (Sec. II A):
 * stage_sweep[i * 33 + k] for window i, -1 for stages not (yet) ended there
 * (h * 33 values).  The sweeps a stage took are the differences between
 * consecutive entries. */
rewl_status rewl_get_stage_sweeps(rewl_ctx *ctx, int inst, int64_t *stage_sweep);

/* Progress: all_converged over all instances; sweeps done; ln f per window of
 * instance `inst` (h values, 0 once converged; may be NULL). */
rewl_status rewl_status_query(rewl_ctx *ctx, int inst, int *all_converged, double *ln_f_per_window,
                              long *sweeps);

/* Warm start: ln g of every walker of instance `inst` from ln_g0 (B values on
 * the instance's bins, rounded to 2^-32), start at ln f = ln_f_start (a power
 * of two), or frozen (pure sampling with weights 1/g, H still counted) if
 * ln_f_start == 0. */
rewl_status rewl_set_initial_lng(rewl_ctx *ctx, int inst, const double *ln_g0, double ln_f_start);

/* Geometry of instance `inst` (any pointer may be NULL): windows h, walkers
 * per window m, bins B, window width w (the widest window: the length of each
 * walker's ln g and H rows), lo[h] = first bin of each window, reach[B] (1 =
 * some configuration has that energy). */
rewl_status rewl_geometry(rewl_ctx *ctx, int inst, int *h, int *m, int *B, int *w, int *lo,
                          uint8_t *reach);

/* Bins of each window of instance `inst` (ww[h]; all equal to w unless the
 * windows were given to rewl_create_batch_windows). */
rewl_status rewl_window_widths(rewl_ctx *ctx, int inst, int32_t *ww);

/* Full walker state of instance `inst` for inspection and parity tests.  Any
 * pointer may be NULL.  spins: [h*m][N] int8 (Ising +-1, Potts 0..q-1) of the
 * configuration each walker slot holds; E, bin: [h*m]; ln_g: [h*m][w] FP64;
 * H: [h*m][w] (uint32, counts modulo 2^32); stage, conv: [h] (conv 0 =
 * running, 1 = converged: ln g frozen and H no longer counted, 2 = sampling
 * with frozen weights set by rewl_set_initial_lng: H counted); latch: [h*m];
 * replica: [h*m] id of the configuration (follows exchanges). */
rewl_status rewl_get_state(rewl_ctx *ctx, int inst, int8_t *spins, int64_t *E, int32_t *bin,
                           double *ln_g, uint32_t *H, int32_t *stage, uint8_t *conv,
                           uint8_t *latch, int64_t *replica);

/* Counters of instance `inst` (any pointer may be NULL): exchange proposals
 * and acceptances per window pair [h], accepted moves per walker [h*m], sweep
 * count at which each window converged [h] (-1: not yet). */
rewl_status rewl_get_counters(rewl_ctx *ctx, int inst, uint64_t *ex_prop, uint64_t *ex_acc,
                              uint64_t *n_accepted, int64_t *conv_sweep);

/* Options.  REWL_OPT_CHECK_EVERY: sweeps between flatness tests (>= 1).
 * REWL_OPT_PRODUCER_WARPS: force the autotuner's producer warps per thread
 * block (0 = auto, 1..4).  REWL_OPT_WINDOWS_PER_CTA: force windows per thread
 * block (0 = auto; at most 32 walkers per block).
 * REWL_OPT_MAX_SWEEPS_PER_LAUNCH: split long rewl_run calls (>= 1).
 * REWL_OPT_AUTOTUNE: 1 (default) = before the first run, time a few launch
 * shapes on a shadow copy of the batch (same descriptors, its own memory) and
 * keep the fastest; 0 = shape rule only.
 * REWL_OPT_LATTICE_PLACEMENT: where the sweep kernel keeps the walkers'
 * lattices while it runs: 0 (default) = shared memory up to 16 KB per walker
 * (Potts L <= 128, Ising L <= 352), global memory above (e.g. the paper's
 * Potts L = 200...400); 1 = always global; 2 = always shared (contexts
 * whose windows' state then exceeds shared memory fail to plan, REWL_EINVAL).
 * Shapes and placement never change results.
 * REWL_OPT_LNG_SHIFT: s in 1..20 (default 20).  ln g of a window is defined
 * up to a constant (the pieces are joined by their differences, Sec. II B;
 * acceptance and Eq. (1) use differences within one window): at each flatness
 * test, a running window whose walkers' ln g has reached 2^s on every
 * realisable bin has 2^s taken off those bins (ln g and its stage-start copy,
 * so H and the trajectory are unchanged).  This keeps ln g inside the exactly
 * representable range |ln g| < 2^21 on large lattices, where the first stages
 * add far more than 2^21 per bin.  Small s is for tests.
 * Launch-shape options may only be set before the first run. */
enum { REWL_OPT_CHECK_EVERY = 1, REWL_OPT_PRODUCER_WARPS = 2, REWL_OPT_WINDOWS_PER_CTA = 3,
       REWL_OPT_MAX_SWEEPS_PER_LAUNCH = 4, REWL_OPT_AUTOTUNE = 5, REWL_OPT_LATTICE_PLACEMENT = 6,
       REWL_OPT_LNG_SHIFT = 7 };
rewl_status rewl_set_option(rewl_ctx *ctx, int option, long value);

/* Number of kernel launches this context enqueued so far (graph replays count
 * each node). */
long rewl_launch_count(const rewl_ctx *ctx);

/* Bytes this context copied host -> device (*h2d) and device -> host (*d2h)
 * since it was created: descriptors and windows at creation, warm-start ln g,
 * checkpoint loads; every read-out, progress poll and error-word check.
 * Copies the caller makes itself are not included.  Either pointer may be
 * NULL; REWL_EINVAL for a NULL context. */
rewl_status rewl_transfer_bytes(const rewl_ctx *ctx, int64_t *h2d, int64_t *d2h);

/* Checkpoint: the complete state (lattices, energies, ln g, H, stages,
 * latches, Philox counters, exchange counter) to a file; loading it resumes
 * bit-exactly. */
rewl_status rewl_save(rewl_ctx *ctx, const char *path);
rewl_status rewl_load(rewl_ctx **out, const char *path, void *cuda_stream);

/* Text of the first error of this context (or of the last failed create when
 * ctx is NULL).  Never NULL. */
const char *rewl_last_error(const rewl_ctx *ctx);

/* Release device memory, graphs and the stream the library created. */
void rewl_destroy(rewl_ctx *ctx);

/* ------------------------------------------------------------------------
 * Learned warm start (not part of the paper's method): a 5 -> 128 -> 128 ->
 * 128 -> 1 perceptron with tanh hidden units predicting the entropy density
 * s = ln g(E) / N from x = (model, 16/L, log10 q, E/N, window / (h-1)).
 * BF16 tensor-core products with FP32 accumulation; FP32 master weights;
 * trained with the mean squared error (loss = mean (y - t)^2 / 2) and Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  It only sets the starting ln g and ln f
 * of Wang-Landau, which then corrects any error of the prediction.
 * Parameter vector (33921 floats): W1 [128x5], b1, W2 [128x128], b2,
 * W3 [128x128], b3, W4 [1x128], b4, W[out][in].
 * x, t, y below are device pointers; n is a multiple of 64, n <= max_batch.
 * ------------------------------------------------------------------------ */
typedef struct rewl_mlp rewl_mlp;

/* Allocate a network with scratch for batches of up to max_batch samples
 * (multiple of 64); weights uniform(+-1/sqrt(fan_in)) from Philox(seed). */
rewl_status rewl_mlp_create(rewl_mlp **out, int max_batch, unsigned long long seed, void *cuda_stream);
rewl_status rewl_mlp_set_params(rewl_mlp *net, const float *host_params, long n);  /* resets Adam */
rewl_status rewl_mlp_get_params(rewl_mlp *net, float *host_params, long n);
/* y[n] = network(x[n][5]). */
rewl_status rewl_mlp_forward(rewl_mlp *net, const float *x, float *y, int n);
/* Gradient of the loss over the batch (host out, 33921 floats) and the loss. */
rewl_status rewl_mlp_gradient(rewl_mlp *net, const float *x, const float *t, int n, float *grad_host,
                              float *loss_host);
/* One Adam step on the batch; loss_host (may be NULL) receives the loss
 * before the step. */
rewl_status rewl_mlp_train_step(rewl_mlp *net, const float *x, const float *t, int n, float lr,
                                float *loss_host);
long rewl_mlp_launch_count(const rewl_mlp *net);
const char *rewl_mlp_last_error(const rewl_mlp *net);
void rewl_mlp_destroy(rewl_mlp *net);

/* Forward pass that allocates nothing (the paper has no counterpart; this is
 * a library service).  For callers that must not allocate device memory once
 * running -- their device memory belongs to another allocator (a framework's
 * caching pool, a budget fixed at start-up) or cudaMalloc's implicit
 * synchronisation of the device is not acceptable where they call from.
 * params: device pointer to the 33921 FP32 parameters (layout above); x: device
 * [n][5]; y: device [n]; n a multiple of 64, at most 1024 (REWL_EINVAL
 * otherwise, message in rewl_mlp_last_error(NULL)).  The activations live in a
 * static device array of 3,276,800 bytes that every GPU loading the library
 * holds until exit; the first call on a device looks up its address there (so
 * make that first call before any stream capture) and keeps it for the rest of
 * the process: after cudaDeviceReset() on that device the kept address is
 * stale, so the entry point must not be called again in that process.  All
 * calls share the array: calls whose work overlaps on the GPU race.
 * Asynchronous on cuda_stream (NULL: the legacy default stream); calls no
 * allocator. */
rewl_status rewl_mlp_forward_noalloc(const float *params, const float *x, float *y, int n, void *cuda_stream);

/* Warm start of instance `inst`: every walker of window i gets
 * ln g(E) = N s(E) (shifted so the window's smallest realisable value is 0,
 * rounded to 2^-32), H = 0, and ln f = ln_f_start (a power of two; 0 freezes). */
rewl_status rewl_warm_start(rewl_ctx *ctx, int inst, rewl_mlp *net, double ln_f_start);

/* Primitive checks (device, for tests).  Acceptance thresholds
 * lam(k) = max(1, trunc(2^32 * -ln((k + 1) 2^-24))) evaluated by the device
 * routine, and Philox4x32-10 blocks for (key, counters).  k, ctr, out: device
 * pointers; n elements (blocks).  Synchronous. */
rewl_status rewl_debug_lam(const uint32_t *k_dev, int64_t *out_dev, long n);
rewl_status rewl_debug_philox(uint32_t key0, uint32_t key1, const uint32_t *ctr_dev,
                              uint32_t *out_dev, long n);

#ifdef __cplusplus
}
#endif
#endif /* REWL_H */

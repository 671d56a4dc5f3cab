/*
 * kx.h -- C ABI of the GB300-native chemistry source-term library.
 *
 * The library evaluates, for one reaction mechanism and a batch of
 * thermochemical states (T, p, Y_k), the quantities of the KinetiX method
 * (arXiv 2411.02640, Appendix A): net species production rates
 * (Sec. A.2), mixture heat capacity and enthalpy (Sec. A.1) and
 * mixture-averaged transport properties (Sec. A.3.5).  kx_load_mechanism
 * reads a mechanism file, emits CUDA C++ specialised to that mechanism and
 * compiles it for sm_103a with NVRTC; the other calls launch the compiled
 * kernels.  By default the production-rate kernels group the reactions
 * into classes of one code shape (kind, reversibility, blend, entry
 * counts) and run one loop per class over per-class constant tables, and
 * the transport kernels loop over per-pair coefficient tables; the
 * alternative native float64 and mixed kernels (kx_options.rates_arith = 1,
 * rates_mode = 1) are fully unrolled with the mechanism's constants as
 * immediates.
 *
 * Conventions shared by every call below:
 *   - Every array argument is a DEVICE pointer to float64 data that the
 *     caller owns and keeps alive until the stream work completes.  State
 *     arrays are structure-of-arrays: T[n] in K, p[n] in Pa and Y[N_s][ld]
 *     (species-major, mass fractions, point index contiguous, ld >= n).
 *     Per-species outputs use the same [N_s][ld] layout.
 *   - Units are SI with kmol: W in kg/kmol, concentrations in kmol/m^3,
 *     production rates in kmol/(m^3 s).
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) and return after enqueueing; a launch failure is
 *     returned at once.  n == 0 is a no-op that returns KX_OK.
 *   - Y need not be normalised: concentrations use
 *     C_k = (p/(R T)) (Y_k/W_k) / sum_j (Y_j/W_j).
 *   - A point with T <= 0, p <= 0 or a non-finite T or p gets NaN in every
 *     output, and so does, in the calls that form concentrations or mole
 *     fractions (all but kx_thermo), a point whose sum_k Y_k/W_k is not
 *     positive and finite; such points are recorded for
 *     kx_last_point_status; nothing traps.  Other non-finite Y propagates
 *     as NaN.
 *   - A handle may be used from several host threads and streams at once.
 *   - Errors: every call returns a kx_status; kx_last_error() gives a
 *     message for the calling thread's last failure.
 */
#ifndef KX_H
#define KX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kx_mech* kx_handle;

typedef enum {
  KX_OK = 0,
  KX_ERR_IO = 1,            /* mechanism file cannot be read */
  KX_ERR_PARSE = 2,         /* malformed mechanism file */
  KX_ERR_UNBALANCED = 3,    /* a reaction does not conserve atoms */
  KX_ERR_ARG = 4,           /* null pointer, bad size or bad option */
  KX_ERR_OOM = 5,           /* host or device allocation failed */
  KX_ERR_COMPILE = 6,       /* NVRTC failed on the emitted source */
  KX_ERR_CUDA = 7,          /* a CUDA runtime call failed */
  KX_ERR_TIMEOUT = 8,       /* a host-side wait ran past its deadline */
  KX_ERR_NONFINITE_INPUT = 9, /* kx_last_point_status: a point was outside the domain */
  KX_ERR_UNSUPPORTED = 10   /* feature not available for this mechanism */
} kx_status;

typedef enum {
  KX_FP64 = 0,   /* float64 ACCURACY: results within 1e-10 of the per-point
                    scale max_k |W_k wdot_k| (production rates) and 1e-12
                    relative (thermo, transport) of a float64 evaluation.
                    By default the arithmetic is double-float -- each value a
                    pair of float32s, about 2^-47 relative per operation, with
                    float32's exponent range, run on the float32 pipe -- and
                    the production rates are formed in log space and
                    accumulated in float pairs under a per-state power-of-two
                    scale, reactions negligible for every state of a warp in
                    float32 (see kx_production_rates); kx_options.rates_arith
                    = 1 selects native float64
                    production rates and rates of progress, tr_mode = 1
                    native float64 transport.  kx_thermo is always
                    double-float. */
  KX_MIXED = 1   /* float32 bulk arithmetic (ln k_f, third body, falloff
                    blend, ln R_f); float pairs for the Gibbs sums of ln K_c;
                    the forward-minus-reverse difference resolved from that
                    ratio and the production-rate accumulation in float64
                    (production rates); float32 mixing rules (transport) */
} kx_precision;

/* Load options; a zero-initialised struct (or NULL) selects the defaults. */
typedef struct {
  int diff_mode;      /* 0 default (symmetric), 1 symmetric pairs (D_kj once per pair; float64-accurate
                        Wilke phi_kj once per pair, phi_jk from phi_kj), 2 full matrices */
  int kc_mode;        /* 0 default (log space: k_r = exp(ln k_f - ln K_c)),
                         1 per-species exp(-G_k/RT) products, one division per reaction */
  int tr_mode;        /* float64 transport: 0 (default) double-float arithmetic on the float32
                         pipe (float64 accuracy, ~2^-47 per operation), 1 native float64 */
  int rates_mode;     /* native float64 and mixed production-rate kernels: 0 (default) automatic --
                         fully unrolled up to 64 species and 400 reactions, table driven beyond;
                         1 unrolled; 2 table driven */
  int rates_arith;    /* arithmetic of the KX_FP64 production rates and rates of progress:
                         0 (default) or 2 double-float (float32 pairs, ~2^-47 per operation) in
                         log space on the float32 pipe, one table-driven loop per reaction class,
                         wdot accumulated in float pairs under a per-state power-of-two scale;
                         1 native float64 */
  int tr_layout;      /* transport kernels' per-thread species vectors: 1 all in shared-memory
                         columns; 2 the mole fractions in local memory (half the shared memory per
                         thread, twice the resident warps); 0 (default) or 3 every vector in local
                         memory (no shared memory; residency set by registers, 64 by default) */
  int maxrreg;        /* register cap per thread for the generated kernels; 0 = compiler choice */
  int block;          /* threads per block; 0 = 128 */
  int lazy;           /* 0: compile the production-rate, thermo and transport kernels at load
                         (in parallel), the rates-of-progress and adjoint kernels on first
                         use; 1: every kernel on first use */
  int verbose;        /* 1: print compile times, registers and local memory per thread to stderr */
  int libmath;        /* 1: CUDA's exp/log in the float64 kernels instead of the library's own */
  int compile_only;   /* 1: emit and compile but do not load onto a device (no GPU needed);
                         launch calls on such a handle return KX_ERR_UNSUPPORTED */
  int rates_layout;   /* double-float KX_FP64 production rates: 0 (default) by batch size -- the
                         warp-cooperative kernel for batches below min(C, 49152 u) states and the
                         thread-per-state kernel from there on, C being the thread-per-state
                         kernel's resident capacity (one wave of its blocks on every SM; ~78k
                         states on GB300 at 128 threads per block) and u the share of lane slots
                         the warp-cooperative class rounds fill (~0.2 for 9/21, ~0.9 for 53/325);
                         the crossover measured on GB300;
                         1 always one thread per state (species vectors in local memory);
                         2 always warp-cooperative (the states of a warp share its lanes: the
                         reactions of each class dealt out as (state, reaction) pairs, species
                         vectors and per-reaction rates in shared memory, wdot gathered
                         species-major).  The two kernels agree to ~1e-11 of the per-point scale,
                         not bit for bit (different summation orders). */
  int rates_group;    /* warp-cooperative production rates: states per warp, a power of two up to
                         32; 0 (default) one */
  int vjp_form;       /* double-float adjoint, the terms d R/d C_k = nu R/C_k: 0 (default) the
                         reaction's rate mantissa times a per-state reciprocal 1/|C_k| (log space
                         only where the rate underflows); 1 one log-space exponential
                         exp(ln |R| - ln |C_k|) per entry (no reciprocal table) */
  int vjp_layout;     /* double-float adjoint: 0 (default) by batch size -- the warp-cooperative
                         kernel for batches below min(C, 8192 w u^2) states, C the thread-per-state
                         kernel's resident capacity, w the warp-cooperative kernel's resident warps
                         per SM and u the share of lane slots its class rounds fill (the crossover
                         measured on GB300: ~8k states for 9/21, ~85k for 53/325, ~32k for
                         160/900), one thread per state from there on; 1 always one thread per
                         state; 2 always warp-cooperative (one state per warp, its vectors and
                         per-reaction terms in shared memory, d/dC_k gathered species-major;
                         mechanisms whose warp slice exceeds 50 KB keep one thread per state
                         under 0 and are refused under 2).  The two agree to ~1e-10 of each
                         entry's term scale, not bit for bit. */
  int rates_negligible; /* double-float KX_FP64 production rates: 0 (default) a reaction whose rate
                         is below 2^-40 of its state's largest, for every state of a warp, is
                         evaluated in float32 (its error is far inside the per-point bar, but a
                         species all of whose reactions are that small gets wdot_k to ~1e-4 of
                         itself); 1 every reaction in float pairs (wdot_k to ~1e-11 of the
                         species' own gross rate, for the species within 1e-40 of their state's
                         largest rate: for finite differences of the rates) */
  const char* cache_dir; /* directory for compiled kernels; NULL = $KX_CACHE_DIR or ~/.cache/kx */
} kx_options;

/* Parse, validate and compile a mechanism (file format KXMECH 1).  On
 * success *out owns the mechanism; free it with kx_free_mechanism. */
kx_status kx_load_mechanism(const char* path, const kx_options* opt, kx_handle* out);

/* Release a handle.  The caller must have synchronised every stream that
 * still has work of this handle in flight. */
kx_status kx_free_mechanism(kx_handle h);

/* Species and reaction counts; W (may be NULL) receives N_s molecular
 * weights in kg/kmol. */
kx_status kx_mechanism_info(kx_handle h, int* n_species, int* n_reactions, double* W);

/* Net production rates wdot[N_s][ld] (Sec. A.2: Eq. (arrhenius), third-body
 * and falloff modifiers Eq. (c_i) and (blend), Eq. (K_p), Eq. (r_i) and the
 * stoichiometric sum wdot_k = sum_i nu_ki R_i).  KX_FP64 with the default
 * double-float kernel evaluates a reaction in float32 when, for every state of
 * a warp (32 consecutive states), its rate is below 2^-40 of that state's
 * largest rate, where float32's error leaves the result far inside the
 * float64 bar: a state's results can therefore differ, within the bar (~1e-11
 * of the per-point scale), with the states it shares a warp with (a call on a
 * sub-range that does not start at a multiple of 32 states, or a batch mixed
 * with other states); the same batch gives the same bits.  A species that
 * only such reactions produce or consume gets its wdot_k to ~1e-4 of itself
 * (still ~1e-16 of the per-point scale); kx_options.rates_negligible = 1
 * evaluates every reaction in float pairs (for finite differences). */
kx_status kx_production_rates(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                              double* wdot, int64_t n, kx_precision precision, void* stream);

/* Rates of progress q[N_r][ld] of every reaction, R_i = c_i r_i (Sec. A.2),
 * the per-reaction quantity the paper validates as "reaction rates"
 * (Table 3). */
kx_status kx_rates_of_progress(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                               double* q, int64_t n, kx_precision precision, void* stream);

/* Mass-based mixture cp[n] in J/(kg K) and h[n] in J/kg from the NASA-7
 * blocks (Sec. A.1: c_p = sum_k Y_k C_p,k / W_k, h = sum_k Y_k H_k / W_k).
 * p is accepted for symmetry and not used. */
kx_status kx_thermo(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                    double* cp, double* hmass, int64_t n, void* stream);

/* Mixture-averaged transport (Sec. A.3.5): Wilke/Bird viscosity mu[n] in
 * Pa s, Mathur conductivity lambda[n] in W/(m K) and diffusion coefficients
 * Dk[N_s][ld] in m^2/s (Eq. (mix_diff)), from the ln T polynomial fits of
 * ln eta_k, ln lambda_k and ln D_kj (Sec. A.3.4), D_kj scaled by p_atm/p.
 * A species whose partners all have X_j = 0 gets its self-diffusion D_kk. */
kx_status kx_transport(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                       double* mu, double* lambda, double* Dk, int64_t n, kx_precision precision, void* stream);

/* The two halves of kx_transport, for callers that need only one of them:
 * Wilke viscosity mu[n] and Mathur conductivity lambda[n]; and the
 * mixture-averaged diffusion coefficients Dk[N_s][ld] (Eq. (mix_diff)). */
kx_status kx_viscosity_conductivity(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                                    double* mu, double* lambda, int64_t n, kx_precision precision, void* stream);
kx_status kx_diffusion(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld, double* Dk,
                       int64_t n, kx_precision precision, void* stream);

/* Vector-Jacobian product of the production rates at fixed p: for each
 * point, gT = sum_k v_k d wdot_k/dT and gY[j] = sum_k v_k d wdot_k/dY_j,
 * with v[N_s][ld] and gY[N_s][ld].  The paper lists the analytical
 * Jacobian as future work (Sec. 4); this is its adjoint form.  Float64
 * accuracy: by default double-float arithmetic on the float32 pipe, each
 * derivative term formed from the log-space rates (so an absent species,
 * Y_k = 0, keeps its exact derivative) and accumulated under a running
 * power-of-two scale of its own; kx_options.rates_arith = 1 selects the
 * native float64 kernel.  One thread per point, or, for batches below the
 * crossover that kx_options.vjp_layout describes, one warp per point. */
kx_status kx_production_rates_vjp(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                                  const double* v, double* gT, double* gY, int64_t n, void* stream);

/* Per-point domain check.  The method is defined for T > 0, p > 0 and a
 * positive, finite sum_k Y_k/W_k (the concentrations of Sec. A.2 and the
 * mole fractions of Sec. A.3.5 divide by it; kx_thermo does not check it);
 * every kernel of a handle gives the points outside that domain NaN
 * outputs and records the smallest such point index (the index within the
 * call's batch).  This call enqueues on `stream` a read of every record of
 * the handle on the current device and their reset, then waits for
 * `stream`: it returns KX_OK with *first_bad_point = -1 if no point was
 * outside the domain since the handle was loaded or last checked, else
 * KX_ERR_NONFINITE_INPUT with the smallest recorded index (over all calls
 * since then; kx_last_error() names it).  Calls on other streams are seen
 * once they have finished: synchronise them first; a call still running on
 * another stream may record its points before or after the reset. */
kx_status kx_last_point_status(kx_handle h, void* stream, int64_t* first_bad_point);

/* Bytes of the library's static device scratch array used by
 * kx_production_rates_noalloc (one array per device that loads the library,
 * held until the process exits). */
#define KX_NOALLOC_SCRATCH_BYTES ((size_t)128 << 20)

/* Net production rates wdot[N_s][ld] in the float-pair (double-float,
 * float64-accurate) arithmetic of kx_production_rates' default kernel,
 * whatever kx_options.rates_arith says, for callers that cannot have device
 * memory allocated while they run: a CFD code that hands all free device
 * memory to its own pool at start-up (a later allocation fails or fragments
 * it), a time step that must not stall on the device-wide synchronisation
 * that cudaMalloc and cudaFree imply, or a fixed-latency loop that must not
 * meet an out-of-memory error in mid-run.  kx_production_rates keeps each
 * state's species vectors in local memory, whose backing the driver may
 * grow at launch; this variant keeps them in one file-scope static
 * __device__ array of KX_NOALLOC_SCRATCH_BYTES and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   - Set-up: the array's device address is looked up (cudaGetSymbolAddress)
 *     once per device, when a handle is loaded with that device current; a
 *     call on another device, or with a handle loaded with opts.lazy, does
 *     the look-up (and, lazily, the kernel's compile and load, which does
 *     allocate) on its first call there: make that first call before any
 *     stream capture and before the caller's no-allocation region.
 *   - Size limit: the grid is capped so that its threads fit the array and
 *     strides over any n; a mechanism whose one block of threads needs more
 *     than the array (24 N_s bytes per thread: more than ~43,000 species)
 *     is rejected with KX_ERR_UNSUPPORTED and a message in kx_last_error().
 *   - Sharing: every call on a device uses the same array, which keeps the
 *     last call's contents (the kernel sets every value it reads before
 *     reading it).  Calls that overlap on the GPU (on streams with no order
 *     between them) race on the array and give wrong results: order them.
 * Pointers, layout, NaN rules and errors otherwise as kx_production_rates;
 * the results match its KX_FP64 results within the same 1e-10 bound of the
 * per-point scale (bit for bit when both run the default float-pair
 * kernel, not when the handle selects native float64 rates).  The paper has no counterpart: this is runtime
 * plumbing around its method. */
kx_status kx_production_rates_noalloc(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld,
                                      double* wdot, int64_t n, void* stream);

/* Per-kernel build facts of a handle, for logs and benchmarks: kernel names
 * are "wdot_fp64", "wdot_mixed", "rop_fp64", "rop_mixed", "thermo",
 * "visc_fp64", "visc_mixed", "diff_fp64", "diff_mixed", "vjp" and
 * "wdot_fp64_noalloc" (the kernel of kx_production_rates_noalloc),
 * "wdot_fp64_wc" (the warp-cooperative production-rate kernel) and
 * "vjp_wc" (the warp-cooperative adjoint of small batches; absent when
 * kx_options.vjp_layout or rates_arith fixes the adjoint kernel).  Any
 * output pointer may be NULL.  registers and local_bytes: per thread, from
 * the compiler's report (local_bytes is the stack frame: local arrays and
 * register spills, the local memory the driver backs for every resident
 * thread).  fp64_ops/fp32_ops/exps: the emitter's per-point operation
 * counts. */
kx_status kx_kernel_info(kx_handle h, const char* kernel, int* registers, int* local_bytes,
                         double* compile_seconds, double* fp64_ops, double* fp32_ops, double* exps);

/* The emitter's per-point operation counts of one kernel, in this order:
 * float64 plain operations (add, mul, fma), float32 plain operations,
 * float64 exp, float64 log, float64 divisions, float32 exp, float32 log,
 * float32 divisions.  counts must hold 8 doubles. */
kx_status kx_kernel_op_counts(kx_handle h, const char* kernel, double* counts);

/* 64-bit FNV-1a hash of a kernel's emitted source: identifies the exact
 * kernel that a profile was taken of. */
kx_status kx_kernel_source_hash(kx_handle h, const char* kernel, uint64_t* hash);

/* The emitted CUDA C++ source of one kernel (for inspection and tests):
 * *len receives its length in bytes; if buf is not NULL, up to cap - 1
 * bytes of it are copied there, followed by a terminating zero. */
kx_status kx_kernel_source(kx_handle h, const char* kernel, char* buf, size_t cap, size_t* len);

/* Outputs of kx_evaluate_host (bit mask). */
#define KX_OUT_WDOT 1
#define KX_OUT_THERMO 2
#define KX_OUT_TRANSPORT 4

/* Device bytes per state that kx_evaluate_host stages per chunk slot (two
 * slots are used): inputs, and the outputs selected by `outputs`. */
int64_t kx_evaluate_host_bytes_per_state(kx_handle h, int outputs);

/* Production rates, thermo and/or transport for states held in HOST memory
 * (pinned for asynchronous copies), pipelined in chunks: the kernels of
 * even chunks run on stream_a and those of odd chunks on a stream of the
 * library (one chunk's last blocks overlap the next chunk's first), while
 * stream_b copies the next chunk's inputs in and another library stream
 * copies finished chunks' outputs out, so both copy directions overlap the
 * arithmetic.  Events order the streams; before the call returns, stream_a
 * and stream_b are made to wait for everything queued on the library's
 * streams.  The library's two streams and eight events are made on a
 * handle's first call on a device and reused by its later calls there (a
 * call running on another host thread at the same time gets a set of its
 * own); kx_free_mechanism releases them.  Chunks hold a whole number of
 * waves of the launched kernels (states that fill every SM's resident
 * blocks once) where the chunk bound allows one; when there are more than
 * two, the first and the last are about a quarter chunk, so that the
 * copy-in and the copy-out that nothing overlaps are short; every chunk
 * starts at a multiple of 256 states, so the results are bit-identical to
 * the single calls on the whole batch.  T, p [n], Y [N_s][ld] are
 * host inputs; wdot [N_s][ldo], cp, hmass, mu, lambda [n] and Dk [N_s][ldo]
 * are host outputs, those not selected by `outputs` may be NULL.
 * `workspace` is caller-owned device memory of `workspace_bytes`; the chunk
 * is the largest that fits two slots of kx_evaluate_host_bytes_per_state
 * bytes per state (at most `max_chunk` states when max_chunk > 0).  Returns
 * after enqueueing on stream_a and stream_b; the caller synchronises both.
 * Arithmetic and error rules as the single calls.  The paper has no
 * counterpart: this is host IO plumbing around its method. */
kx_status kx_evaluate_host(kx_handle h, const double* T, const double* p, const double* Y, int64_t ld, double* wdot,
                           double* cp, double* hmass, double* mu, double* lambda, double* Dk, int64_t ldo, int64_t n,
                           kx_precision precision, int outputs, void* workspace, size_t workspace_bytes,
                           int64_t max_chunk, void* stream_a, void* stream_b);

/* Copy `rows` rows of n float64 values between host (pinned or pageable)
 * and device buffers with leading dimensions dst_ld and src_ld (in
 * elements), asynchronously on `stream`, in one call: staging of strided
 * state arrays for the serving loop.  The paper has no counterpart; it is
 * host plumbing around the method. */
kx_status kx_copy_rows_async(void* dst, int64_t dst_ld, const void* src, int64_t src_ld, int64_t rows, int64_t n,
                             void* stream);

/* Arithmetic-pipe probe for the roofline denominators (the paper has no
 * counterpart; it measures the machine, not the method): launches `blocks`
 * blocks of `threads` threads (a multiple of 32, at most 256) that each run
 * eight independent chains of `iters` operations of kind `op`: 0 float64
 * FMA, 1 float32 FMA, 2 float32 base-2 exponential on the special-function
 * unit (ex2.approx), 3 CUDA's float64 exp, 4 CUDA's float64 log (plus one
 * add), 5 float64 division (plus one add).  `sink` is a device buffer of
 * blocks * threads doubles that receives the chains' results; *ops (may be
 * NULL) gets the number of operations launched (8 iters blocks threads).
 * Asynchronous on `stream`; the caller times it with events on that stream.
 * Returns KX_ERR_ARG for a bad argument, KX_ERR_CUDA if the launch fails. */
kx_status kx_probe_pipe(int op, int64_t iters, int blocks, int threads, double* sink, void* stream, double* ops);

const char* kx_status_string(kx_status s);

/* Message of the calling thread's last failed call (empty if none). */
const char* kx_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KX_H */

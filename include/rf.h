/*
 * rf.h -- C ABI of the GB300 batched unbinned-likelihood library.
 *
 * The library evaluates, on one GPU, the likelihood of a PDF computation graph
 * over every event of an unbinned dataset, as in "Making RooFit Ready for
 * Run 3" (Hageboeck & Moneta, arXiv:2003.12861):
 *   - Sec. 1: a model is a graph of observables, parameters, functions and
 *     PDFs; every node evaluates to a real value; the top PDF gives the
 *     probability of an event.
 *   - Sec. 4: a likelihood needs the probability of each event; constant
 *     (parameter-only) branches are computed once per parameter point; PDFs
 *     are normalised; Sec. 4.1/4.2 evaluate all events of a node in one call
 *     and reduce with simple reductions.
 * NLL(theta) = -sum_i log( pdf(x_i; theta) / norm(theta) ), its gradient in
 * the free parameters, fits (Sec. 1: "perform fits to data") and toy datasets
 * (Sec. 1: RooStats toy Monte Carlo) are the calls below.
 *
 * Conventions (all calls):
 *   - Every call returns rf_status; nothing throws across the ABI.  On error,
 *     rf_last_error() returns a thread-local message.
 *   - The caller owns every array it passes.  Host arrays are only read (or
 *     written) during the call.  Handles (rf_model, rf_data, rf_mlp) are owned
 *     by the library until the caller destroys them.
 *   - Device pointers borrowed by rf_data_upload(cols_on_device=1) must stay
 *     valid until rf_data_destroy.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - A handle is not thread-safe; distinct handles may be used from
 *     different threads.
 *   - Parameter vectors `theta` hold the FREE parameters in the order of the
 *     PARAM nodes with is_free = 1; n_sets x n_free, row-major.
 */
#ifndef RF_H
#define RF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RF_OK = 0,
  RF_E_INVALID = 1,       /* bad argument, bad graph, size beyond a limit      */
  RF_E_OOM = 2,           /* device or host allocation failed                  */
  RF_E_CUDA = 3,          /* a CUDA runtime call failed                        */
  RF_E_DOMAIN = 4,        /* pdf <= 0 / not finite for some event, or theta
                             outside a pdf's domain; that set's NLL is +inf    */
  RF_E_NOT_CONVERGED = 5, /* a fit stopped before its tolerance                */
  RF_E_TIMEOUT = 6        /* a bounded device wait gave up                     */
} rf_status;

/* Node kinds (Sec. 1: observables, parameters, functions/PDFs). */
typedef enum {
  RF_OBS = 0,      /* observable: lo/hi = range; its column = order among OBS nodes   */
  RF_PARAM = 1,    /* parameter: value = default (fit start), lo/hi = fit bounds;
                      is_free = 0 makes it a constant                                 */
  RF_GAUSS = 2,    /* in = [obs, mu, sigma]           exp(-(x-mu)^2 / 2 sigma^2)      */
  RF_EXP = 3,      /* in = [obs, c]                   exp(c x)                        */
  RF_GAUSSEXP = 4, /* in = [obs, tau, mu, sigma]      exp(-t/tau) (t >= 0) convolved
                      with a unit-area Gaussian(mu, sigma)  (Fig. 1: a convolution)   */
  RF_CHEB = 5,     /* in = [obs, c1..cn], n <= 7      1 + sum c_k T_k(x'), x' = the
                      range mapped to [-1, 1]                                         */
  RF_POLY = 6,     /* in = [obs, a1..an], n <= 7      1 + sum a_k x^k (Fig. 1)        */
  RF_SUM = 7,      /* in = [pdf_1..pdf_n, f_1..f_{n-1}], 2 <= n <= 4: sum f_j pdf_j
                      with f_n = 1 - sum f_j; each pdf_j normalised on its own;
                      all components over the same observables                        */
  RF_PROD = 8,     /* in = [pdf_1..pdf_n], n <= 8, over disjoint observables          */
  RF_POISSON = 9,  /* in = [obs, lambda]  lambda^k exp(-lambda) / k!, k = floor(x)
                      (at most hi-1): the count as a step density of unit steps on
                      an observable range with integer bounds 0 <= lo < hi <=
                      lo + 1e5; normalised by the Poisson mass of k = lo..hi-1
                      (Sec. 4.1 lists the batched Poisson PDF)                        */
  RF_EXTEND = 10,  /* root only, in = [pdf, nu]: extended likelihood, the NLL of a
                      dataset of N events gains nu - N log nu (the Poisson
                      probability of N given the expected count nu, without the
                      constant log N!); nu <= 0 is outside the domain              */
  RF_EXPR = 11     /* in = [obs, p_1..p_n], n <= 7: a density given as a short
                      postfix program over x, p_j and constants (rf_expr, passed
                      to rf_model_create_expr), for PDFs that have no built-in
                      kind (Sec. 5: a fall-back implementation for PDFs that
                      have not been given batch code).  Evaluated per event by
                      the FP64 graph interpreter with its parameter derivatives
                      by forward mode; normalised per parameter point by
                      adaptive 15-point Gauss-Kronrod quadrature on the device
                      (to ~1e-14 of the integral, at most 256 panels per
                      refinement level).  The program must be positive and
                      finite on the range; where it is not, that event (or,
                      in the normalisation, the parameter point) is outside
                      the domain                                               */
} rf_kind;

/* Operations of an RF_EXPR program: one int32 per operation, code | (arg <<
 * 8).  RF_EX_X pushes the observable, RF_EX_PAR pushes the node's parameter
 * arg (input 1 + arg), RF_EX_CONST pushes constant arg; ADD SUB MUL DIV POW
 * pop b then a and push a op b (POW: a^b, a > 0); NEG EXP LOG pop a and push
 * -a, exp(a), log(a) (a > 0). */
typedef enum {
  RF_EX_X = 0, RF_EX_PAR = 1, RF_EX_CONST = 2, RF_EX_ADD = 3, RF_EX_SUB = 4, RF_EX_MUL = 5, RF_EX_DIV = 6,
  RF_EX_NEG = 7, RF_EX_EXP = 8, RF_EX_LOG = 9, RF_EX_POW = 10
} rf_expr_code;

typedef enum { RF_F64 = 0, RF_F32 = 1 } rf_dtype;

/* One graph node.  Every PDF is normalised by its analytic integral over its
 * observable's range [lo, hi] (Sec. 4: normalisation of PDFs). */
typedef struct {
  int32_t kind;   /* rf_kind */
  int32_t n_in;   /* number of valid entries in `in` */
  int32_t in[8];  /* input node indices */
  double value;   /* PARAM: default value */
  double lo, hi;  /* OBS: range; PARAM: bounds (lo >= hi: unbounded) */
  int32_t is_free;/* PARAM: 1 = free parameter */
} rf_node;

typedef struct rf_model rf_model;
typedef struct rf_data rf_data;
typedef struct rf_mlp rf_mlp;

/* ------------------------------------------------------------------ models */

/* Validate a node list and compile it: topological order of the PDFs under
 * `root`, observables bound to columns, free-parameter indices, the
 * per-parameter-point plan (normalisation integrals, Sec. 4) and the
 * per-event program of the fused kernel.  Limits: <= 64 nodes, <= 24 PDF
 * nodes, <= 16 free parameters, <= 8 observables.  RF_E_INVALID on a graph
 * the library cannot evaluate (cycle, PROD factors sharing an observable, SUM
 * components over different observables, wrong arity, limits). */
rf_status rf_model_create(const rf_node* nodes, int32_t n, int32_t root, rf_model** out);

/* The program of one RF_EXPR node: n_ops operations (1..64), n_consts
 * constants (0..16).  A program is checked as a whole: every argument in
 * range, the stack (depth <= 16) never underflows, exactly one value left.
 * Per model at most 128 operations and 32 constants over all its programs. */
typedef struct {
  int32_t node;          /* index of the RF_EXPR node in the node list */
  int32_t n_ops;
  const int32_t* ops;    /* rf_expr_code | (arg << 8) */
  int32_t n_consts;
  const double* consts;
} rf_expr;
/* rf_model_create for a node list with RF_EXPR nodes: exprs[0..n_exprs)
 * gives every RF_EXPR node its program (host arrays, copied).  RF_E_INVALID
 * for an RF_EXPR node without a program, a program given twice or for a
 * node of another kind, or an invalid program. */
rf_status rf_model_create_expr(const rf_node* nodes, int32_t n, int32_t root, const rf_expr* exprs,
                               int32_t n_exprs, rf_model** out);
void rf_model_destroy(rf_model* m);
int32_t rf_model_n_free(const rf_model* m);
int32_t rf_model_n_obs(const rf_model* m);
/* on = 1: evaluate every event of this model with the FP64 graph interpreter
 * (Sec. 4: the likelihood in double precision, node by node per event)
 * instead of the float-float event program of a recognised graph shape;
 * on = 0 (the default) restores the specialised program.  Results agree
 * within the library's stated tolerances either way. */
rf_status rf_model_set_fp64(rf_model* m, int32_t on);
/* Writes a short description of the compiled event program (which fused
 * kernel it runs on) into buf (NUL-terminated, at most cap bytes). */
rf_status rf_model_describe(const rf_model* m, char* buf, int32_t cap);

/* ------------------------------------------------------------------- data */

/* Structure-of-arrays event columns, one per observable (Sec. 4.1: arrays of
 * all entries instead of single values).  cols[c] points to n_events values of
 * type dtype[c] (dtype NULL = all RF_F64).  Ragged sets (toy datasets):
 * offsets[0..n_sets] with offsets[0] = 0 and offsets[n_sets] = n_events
 * (offsets NULL and n_sets = 1 for one dataset).  cols_on_device = 0: host
 * arrays, copied into library-owned device memory; = 1: borrowed (not
 * copied) device, managed or pinned host memory -- pinned host columns are
 * read in place by the kernels over the host link, so no copy precedes a
 * pass; other host memory is refused with RF_E_INVALID.  Events are kept in
 * the given order. */
rf_status rf_data_upload(const rf_model* m, const void* const* cols, const int32_t* dtype, int64_t n_events,
                         const int64_t* offsets, int32_t n_sets, int32_t cols_on_device, rf_data** out);
void rf_data_destroy(rf_data* d);
int64_t rf_data_n_events(const rf_data* d);
int32_t rf_data_n_sets(const rf_data* d);
/* Copy events [i0, i1) of column `col` to host memory, widened to double. */
rf_status rf_data_read(const rf_data* d, int32_t col, int64_t i0, int64_t i1, double* out);
/* Copy the n_sets + 1 set offsets to host memory. */
rf_status rf_data_offsets(const rf_data* d, int64_t* out);

/* ------------------------------------------------------------- likelihood */

/* NLL of every set: nll[s] = -sum_{i in set s} log p_i(theta_s) (Sec. 4:
 * "the probability of observing each event"), non-extended.  theta and nll
 * are HOST arrays (n_sets x n_free, n_sets).  The sum is deterministic: it
 * is a fixed tree over 4096-event chunks (in-chunk lane sums, then
 * compensated two-sum merges), independent of launch shape.  A set with an
 * event whose pdf is <= 0 or not finite gets nll = +inf and the call returns
 * RF_E_DOMAIN.  Synchronous on `stream`. */
rf_status rf_nll(const rf_model* m, const rf_data* d, const double* theta, double* nll, void* stream);

/* NLL and its gradient in the free parameters, from one pass over the events
 * (adjoint of the graph in the same kernel).  grad: HOST, n_sets x n_free. */
rf_status rf_nll_grad(const rf_model* m, const rf_data* d, const double* theta, double* nll, double* grad,
                      void* stream);

/* Device-resident, asynchronous form of rf_nll_grad for CUDA-graph capture
 * and pipelines: d_theta (n_sets x n_free) and d_out (n_sets x (1 + n_free):
 * nll then gradient) are DEVICE pointers; d_flags (n_sets int32, device)
 * receives the count of events with pdf <= 0 / not finite.  Launches only;
 * never synchronises or allocates after the first call for this (m, d). */
rf_status rf_nll_grad_async(const rf_model* m, const rf_data* d, const double* d_theta, double* d_out,
                            int32_t* d_flags, void* stream);

/* Per-chunk partial sums (the first level of the reduction), for checking a
 * sample of chunks against an independent evaluation: for chunk c of set
 * `set` (4096 events each, the last one ragged), out[c*(1+n_free)] = the sum
 * of log p_i over the chunk and out[c*(1+n_free)+1+k] = the sum of
 * dlog p_i/dtheta_k, for at most max_chunks chunks.  *n_chunks receives the
 * set's chunk count. */
rf_status rf_nll_chunks(const rf_model* m, const rf_data* d, const double* theta, int32_t set, double* out,
                        int32_t max_chunks, int32_t* n_chunks);

/* Launch shape of the fused event kernel.  Its block is always 128 threads:
 * lane l of a block sums events l, l + 128, ... of a chunk, and that fixed
 * lane-to-event map is what makes the NLL independent of the launch
 * (bitwise), so threads_per_block accepts 0 or 128 only.  The tunable
 * dimension is blocks_per_sm, the resident blocks per SM of the persistent
 * grid (1..32; 0 = library choice).  The work unit (a whole 4096-event chunk,
 * or a quarter chunk for datasets of fewer than 1024 chunks) is fixed by
 * the dataset for the same reason. */
rf_status rf_set_launch(rf_model* m, int32_t threads_per_block, int32_t blocks_per_sm);

/* Autotuner: times `passes` NLL+gradient passes over `d` for every resident
 * block count per SM that fits the kernel's registers and shared memory
 * (from {1..8, 12, 16}), keeps the fastest on the model (as rf_set_launch
 * would) and reports it: *threads_per_block = 128, *blocks_per_sm, *best_ms
 * the mean pass time of the winner.  Results do not depend on the choice
 * (bitwise). */
rf_status rf_autotune(rf_model* m, rf_data* d, int32_t passes, int32_t* threads_per_block, int32_t* blocks_per_sm,
                      double* best_ms);
/* The same search, reporting the whole grid: for each candidate i < *n
 * (at most cap), blocks_per_sm[i] and its mean pass time ms[i]; the winner
 * is kept on the model. */
rf_status rf_autotune_scan(rf_model* m, rf_data* d, int32_t passes, int32_t cap, int32_t* blocks_per_sm, double* ms,
                           int32_t* n);

/* ------------------------------------------------------------------- fits */

typedef struct {
  double tol_edm;       /* stop when EDM = g^T H g / 2 < tol_edm (default 1e-7)   */
  int32_t max_evals;    /* per set (default 1000)                                 */
  int32_t want_cov;     /* 1: covariance from the Hessian at the minimum          */
  int32_t no_graph;     /* 1: launch each evaluation directly instead of replaying
                           the captured CUDA graph of the evaluation step; every
                           quasi-Newton step then runs on the host               */
  int32_t host_steps;   /* 1: every quasi-Newton step on the host.  0 (default):
                           in a fit of two or more sets, once fewer than 2^23
                           of their events are still being fitted, the rounds
                           run on the device, the step included, 8 per graph
                           launch; the trial points, and so the results, are
                           bitwise those of host steps                           */
} rf_fit_opts;

/* Maximum-likelihood fit of every set (Sec. 1: fits).  Quasi-Newton (BFGS)
 * over internal coordinates (bounded parameters through
 * theta = lo + (hi-lo)(sin phi + 1)/2), strong-Wolfe line search; every
 * evaluation of all still-active sets is one device pass (n_sets > 1: the
 * batched toy fit).  The steps run on the host while many events are being
 * fitted, then on the device (see rf_fit_opts.host_steps), with the same
 * results.  theta0: HOST n_sets x n_free or NULL (the PARAM
 * defaults).  Outputs (HOST): theta_hat (n_sets x n_free), nll_min (n_sets),
 * cov (n_sets x n_free^2, or NULL), n_evals (n_sets), fit_status (n_sets:
 * rf_status per set).  Returns RF_OK when the call ran, even if some sets did
 * not converge (see fit_status). */
rf_status rf_fit(const rf_model* m, const rf_data* d, const double* theta0, const rf_fit_opts* opts,
                 double* theta_hat, double* nll_min, double* cov, int32_t* n_evals, int32_t* fit_status);

/* rf_fit for the sets sets[0..n) of d only (distinct indices in
 * [0, n_sets)), fitted together as one batch: theta0 (HOST n x n_free, or
 * NULL for the defaults) and the outputs are per listed set, in the list's
 * order.  The other sets are not evaluated.  For refitting a few toys of a
 * batch without moving their events. */
rf_status rf_fit_sets(const rf_model* m, const rf_data* d, const int32_t* sets, int32_t n, const double* theta0,
                      const rf_fit_opts* opts, double* theta_hat, double* nll_min, double* cov, int32_t* n_evals,
                      int32_t* fit_status);

/* ------------------------------------------------------------------- toys */

/* Generate n_sets toy datasets on the device (Sec. 1: toy Monte Carlo).
 * theta: HOST, n_sets x n_free if theta_per_set, else one vector for all sets
 * (NULL = defaults).  mean_n: HOST, n_sets expected sizes; poisson = 1 draws
 * N_s ~ Poisson(mean_n[s]) (PTRS of Hoermann 1993 for mean >= 10, inversion
 * below), poisson = 0 uses round(mean_n[s]).  Events are drawn by
 * accept-reject, independently for each factor of a PROD at the root, from
 * Philox4x32-10 (Salmon et al., SC'11) with key = (seed, seed >> 32) and
 * counter = (event, attempt, set, factor); the Poisson draw uses counter
 * (iteration, 0, set, 0xFFFFFFFF).  dtype: per column (NULL = RF_F64); an
 * RF_F32 column stores the double draw rounded to float.  *out is a new
 * rf_data owning its device memory. */
rf_status rf_generate_toys(const rf_model* m, const double* theta, int32_t theta_per_set, uint64_t seed,
                           int32_t n_sets, const double* mean_n, int32_t poisson, const int32_t* dtype,
                           rf_data** out);

/* Per-set 64-bin histogram of column `col` over its observable range,
 * normalised by the set's event count: bin = floor((x - lo) * (64/(hi - lo))),
 * clamped to [0, 63].  d_out: DEVICE float, n_sets x 64. */
rf_status rf_hist64(const rf_model* m, const rf_data* d, int32_t col, float* d_out, void* stream);

/* ------------------------------------------------------------ learned start */

/* A multilayer perceptron that maps the 64-bin histogram of a toy dataset
 * (rf_hist64) to a starting point for its fit.  The paper has no learned
 * component; this is the learned-start configuration: n_in inputs,
 * n_hidden_layers hidden layers of n_hidden GELU (erf form) units, n_out
 * linear outputs.  GEMM operands are rounded to BF16 (nearest even) and
 * multiplied on the fifth-generation tensor cores (tcgen05) with FP32
 * accumulation in tensor memory; master weights are FP32.  A GEMM whose
 * wait for its tensor-core work gives up (bounded) makes the next
 * synchronous call (rf_mlp_grad with a loss, rf_mlp_train, rf_mlp_predict)
 * return RF_E_TIMEOUT.  Weights start Uniform(+-1/sqrt(fan_in)) from
 * `seed`, biases 0.
 * Parameters (flat FP32): per layer W[n_in x n_out] row-major, then b[n_out]. */
rf_status rf_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_hidden_layers, int32_t n_out, uint64_t seed,
                        rf_mlp** out);
void rf_mlp_destroy(rf_mlp* n);
int64_t rf_mlp_n_params(const rf_mlp* n);
rf_status rf_mlp_get_params(const rf_mlp* n, float* host);        /* n_params FP32 master weights */
rf_status rf_mlp_set_params(rf_mlp* n, const float* host);
/* d_y[batch x n_out] = net(d_x[batch x n_in]); DEVICE pointers, asynchronous.
 * After rf_mlp_train with standardise = 1 the outputs are mapped back to
 * the targets' units (output * sd + mean). */
rf_status rf_mlp_forward(rf_mlp* n, const float* d_x, int32_t batch, float* d_y, void* stream);
/* Forward + backward of the mean-squared error against d_t (DEVICE,
 * batch x n_out, in the net's raw output units); *loss (host, may be NULL;
 * synchronises when given) and the gradient kept inside the net for
 * rf_mlp_adam, and copied to d_grad (DEVICE, n_params floats) if not NULL. */
rf_status rf_mlp_grad(rf_mlp* n, const float* d_x, const float* d_t, int32_t batch, float* loss, float* d_grad,
                      void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient. */
rf_status rf_mlp_adam(rf_mlp* n, float lr, void* stream);
/* Train on rows x (n_in, n_out) DEVICE arrays: `epochs` passes of shuffled
 * mini-batches (seeded permutation, the ragged remainder dropped), Adam with
 * a cosine decay of the learning rate from lr to 0; standardise = 1 trains
 * on per-output standardised targets and keeps the affine map for
 * rf_mlp_forward.  *final_loss = the mean loss of the last epoch. */
rf_status rf_mlp_train(rf_mlp* n, const float* d_x, const float* d_t, int32_t rows, int32_t batch, int32_t epochs,
                       float lr, uint64_t seed, int32_t standardise, float* final_loss);
/* Checkpoint: dimensions, step, master weights, Adam moments, output map. */
/* The learned fit start (the network's use): for every set of d, the
 * 64-bin histogram of observable col (rf_hist64), the network's forward
 * pass (with the output de-standardisation of rf_mlp_train), and the
 * prediction in theta0 (HOST, n_sets x n_free doubles, the model's free
 * parameters in order; a start for rf_fit).  A bounded parameter's
 * prediction is kept 5 % of its range inside the bounds (at a bound the
 * fit's bound transform is stationary and the parameter barely moves).
 * The network must map 64 inputs to the model's n_free outputs
 * (RF_E_INVALID otherwise).  Synchronous. */
rf_status rf_mlp_predict(rf_mlp* n, const rf_model* m, const rf_data* d, int32_t col, double* theta0);
rf_status rf_mlp_save(const rf_mlp* n, const char* path);
rf_status rf_mlp_load(const char* path, rf_mlp** out);

/* rf_nll_grad with the events coming from HOST memory: host_cols (n_obs
 * pointers, the dataset's layout and dtypes) are copied into the dataset's
 * library-owned device columns and evaluated in one call -- the whole
 * data path of a fit whose events live in host memory.  The work items are
 * cut into up to 8 segments of >= 512 Ki events (the last two a half and a
 * quarter of the others);
 * segment k's copy (on the
 * library's copy stream) overlaps the event passes over earlier segments
 * (on four library compute streams that start after the parameter-point
 * kernel on `stream` and that `stream` waits for), so the call takes about
 * the copy time plus one segment's pass.
 * Pinned host memory is required for the overlap (pageable memory works,
 * serialised).  nll, grad: HOST as in rf_nll_grad.  Returns after the
 * results are on the host.  RF_E_INVALID for a dataset that borrows its
 * columns. */
rf_status rf_nll_grad_stream(const rf_model* m, rf_data* d, const void* const* host_cols, const double* theta,
                             double* nll, double* grad, void* stream);

/* ---------------------------------------------------- binned likelihood */

/* Binned models built from histograms (Sec. 3: HistFactory -- channels of
 * samples with +-1 sigma systematic histograms).  Samples s cover contiguous
 * bins [bin0[s], bin0[s] + nbins[s]) with nominal rates (concatenated in
 * sample order); modifiers tie a sample to one parameter theta_k:
 *   RF_MOD_NORMFACTOR  nu *= theta_k (typically a free, unconstrained scale)
 *   RF_MOD_NORMSYS     nu *= exp(a alpha + b g(alpha)), a, b = (log k_hi -+
 *                      log k_lo) / 2
 *   RF_MOD_HISTOSYS    nu += a_i alpha + b_i g(alpha) bin by bin, before the
 *                      factors, a_i = (h_hi - h_lo)/2, b_i = (h_hi + h_lo)/2 -
 *                      h; h_lo then h_hi (nbins each) follow in hist_data in
 *                      modifier order
 * with g = alpha^2 for |alpha| <= 1, 2|alpha| - 1 beyond: quadratic
 * interpolation between the -1, 0, +1 sigma points and linear extrapolation
 * (in log for normsys), continuous with its first derivative.
 * nu_b = sum over the samples on bin b; for bin counts n_b
 *   NLL = sum_b (nu_b - n_b log nu_b) + sum_{constrained k} theta_k^2 / 2
 * (Poisson terms without log n_b!, unit-Gaussian constraints without their
 * normalisation).  Limits: 8192 bins, 2048 samples (and the block's shared
 * memory: 8 bytes x (2 samples + bins + 256)).  Host arrays are copied. */
typedef enum { RF_MOD_NORMFACTOR = 0, RF_MOD_NORMSYS = 1, RF_MOD_HISTOSYS = 2 } rf_modifier_kind;
typedef struct {
  int32_t sample, kind, param; /* rf_modifier_kind */
  double k_lo, k_hi;           /* RF_MOD_NORMSYS factors (> 0) */
} rf_modifier;
typedef struct rf_binned rf_binned;
rf_status rf_binned_create(int32_t n_bins, int32_t n_samples, const int32_t* bin0, const int32_t* nbins,
                           const double* nominal, int32_t n_params, const int32_t* constrained, int32_t n_mods,
                           const rf_modifier* mods, const double* hist_data, rf_binned** out);
void rf_binned_destroy(rf_binned* m);
int32_t rf_binned_n_params(const rf_binned* m);
/* NLL and gradient of n_sets datasets at once (one parameter point each):
 * counts HOST n_sets x n_bins, theta HOST n_sets x n_params, nll HOST n_sets,
 * grad HOST n_sets x n_params.  A dataset with some nu_b <= 0 gets NLL +inf
 * and the call returns RF_E_DOMAIN.  Deterministic (fixed summation order). */
rf_status rf_binned_nll_grad(rf_binned* m, int32_t n_sets, const double* counts, const double* theta, double* nll,
                             double* grad);
/* The same on DEVICE arrays, asynchronous on `stream`: d_out n_sets x (1 +
 * n_params) (NLL then gradient), d_flags n_sets (1 = some nu_b <= 0). */
rf_status rf_binned_nll_grad_async(rf_binned* m, int32_t n_sets, const double* d_counts, const double* d_theta,
                                   double* d_out, int32_t* d_flags, void* stream);
/* Maximum-likelihood fits of n_sets binned datasets at once (the batched
 * BFGS of rf_fit, one device launch per round over the active datasets):
 * counts HOST n_sets x n_bins, theta0 HOST n_sets x n_params (starts), lo/hi
 * HOST n_params bounds (lo >= hi: unbounded), results as rf_fit. */
rf_status rf_binned_fit(rf_binned* m, int32_t n_sets, const double* counts, const double* theta0, const double* lo,
                        const double* hi, const rf_fit_opts* opts, double* theta_hat, double* nll_min, double* cov,
                        int32_t* n_evals, int32_t* fit_status);
/* Expected counts nu_b (DEVICE n_sets x n_bins) at DEVICE theta, for toys. */
rf_status rf_binned_expected(rf_binned* m, int32_t n_sets, const double* d_theta, double* d_nu, void* stream);

/* ------------------------------------------------------------ measurement */

/* Re-copy host columns (same count and dtypes as the dataset was created
 * with) into a dataset's library-owned device columns, asynchronously on
 * `stream`: the next batch of events in the same layout.  Pinned host memory
 * gives full copy bandwidth.  RF_E_INVALID for a dataset that borrows its
 * columns. */
rf_status rf_data_refill(rf_data* d, const void* const* cols, void* stream);

/* Kernel timing: while enabled (enable = 1), the library brackets every
 * launch of its fused event kernel with CUDA events on the launching stream.
 * rf_kernel_time reads (and with reset = 1 clears) the summed duration in ms
 * and the number of launches since the last reset; it synchronises on the
 * recorded events. */
rf_status rf_kernel_timing(int32_t enable);
rf_status rf_kernel_time(double* total_ms, int64_t* launches, int32_t reset);

/* Number of the library's kernels launched so far in this process (every
 * kernel of the likelihood, fit, generation, histogram and network paths;
 * a replayed evaluation graph counts its kernels; launches recorded into a
 * stream capture are not counted; the roofline probes are not counted).
 * Read it before and after a region to count that region's launches. */
rf_status rf_launch_count(int64_t* n);

/* Events that took the slow path (the decay-resolution convolution near the
 * resolution region) in the last pass over `d`, summed over sets. */
rf_status rf_slow_events(const rf_data* d, int64_t* count);

/* Throughput probes for the roofline, run on the current device:
 *   kind 0: FP64 fused multiply-add rate            -> *rate in FLOP/s
 *   kind 1: FP32 fused multiply-add rate            -> *rate in FLOP/s
 *   kind 2: per-event transcendental set on register data, with CUDA's
 *           FP64 functions (the generic kernel's): n_exp exponentials, n_erfc
 *           complementary error functions, n_log logarithms and n_rcp
 *           reciprocals per event                   -> *rate in events/s
 *   kind 3: streaming read of a device buffer       -> *rate in bytes/s
 *   kind 4: as kind 2 with the library's float-float implementations
 *           (exp, erfcx for erfc, log, reciprocal)  -> *rate in events/s
 *   kind 5: streaming read of pinned host memory by the SMs, in place over
 *           the host link                           -> *rate in bytes/s
 *   kind 6: float-float multiply-add rate (a b + c on float pairs, the
 *           library's ff_fma)                       -> *rate in multiply-adds/s
 * Each probe allocates and frees its own scratch. */
rf_status rf_probe(int32_t kind, int32_t n_exp, int32_t n_erfc, int32_t n_log, int32_t n_rcp, double* rate);

/* Elementwise evaluation of the library's float-float elementary functions
 * (fn 0 exp, 1 log, 2 reciprocal, 3 erfcx) and of CUDA's FP64 ones (fn 10
 * exp, 11 log, 12 reciprocal, 13 erfcx) on DEVICE arrays of n doubles, for
 * validating the former against the latter.  A float-float result outside
 * the function's working range is NaN. */
rf_status rf_math_eval(int32_t fn, const double* d_x, double* d_y, int64_t n, void* stream);

/* ----------------------------------------------------- sharded evaluation */

/* The likelihood is a sum over independent events (Sec. 4), so one dataset
 * can be split over several GPUs -- one process each -- and the shards' sums
 * combined in one exchange step (Sec. 5 names parallelisation as the next
 * step).  Shards are contiguous: rf_shard splits n items (events of one
 * set, or the sets of a toy batch) into `world` ranges whose boundaries are
 * multiples of `align` (use 4096, the reduction's chunk, for events; 1 for
 * sets): rank r gets [*lo, *hi), floor(r C / world) .. floor((r+1) C /
 * world) in units of align, C = ceil(n / align), the last range ending at n.
 * Ranges are disjoint and cover [0, n).  Host only; RF_E_INVALID for n < 0,
 * align < 1, world < 1 or rank outside [0, world). */
rf_status rf_shard(int64_t n, int64_t align, int32_t rank, int32_t world, int64_t* lo, int64_t* hi);

/* One shard's partial sums: as rf_nll_grad_async, but d_pairs (DEVICE,
 * n_sets x (1 + n_free) x 2 doubles) receives per set the compensated pairs
 * (sum, compensation) of sum_i log p_i and of sum_i d log p_i / d theta_k
 * (not negated; a free parameter's slots merged in slot order), and d_flags
 * (DEVICE, n_sets int32) the bad-event count (+2^30 if theta is outside a
 * pdf's domain).  Launches only. */
/* (Not for extended models, whose term needs the whole dataset's size:
 * RF_E_INVALID.) */
rf_status rf_nll_grad_partial(const rf_model* m, const rf_data* d, const double* d_theta, double* d_pairs,
                              int32_t* d_flags, void* stream);

/* The exchange step: merges the shards' pairs in rank order 0 .. world-1
 * with exact two-sum merges (so the result is fixed by the shard layout,
 * independent of which rank's message arrived first) and finishes each set:
 * out[s x (1+n_free)] = NLL = -(s + c) (+inf when flagged), then the
 * gradient -(s + c).  pairs: HOST, world x n_sets x (1 + n_free) x 2;
 * flags: HOST, world x n_sets; flags_out: HOST, n_sets (bad-event counts
 * summed, +2^30 if any shard flagged the domain).  Host only; returns
 * RF_E_DOMAIN when some set is flagged. */
rf_status rf_combine_partials(const double* pairs, const int32_t* flags, int32_t world, int32_t n_sets,
                              int32_t n_free, double* out, int32_t* flags_out);

/* --------------------------------------------------- allocation-free pass */

/* rf_nll_grad_async for one dataset whose columns are caller-owned device
 * arrays, allocating no device memory at all.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc while they run (an online
 * filter or service that reserves all GPU memory at start-up, where an
 * allocation mid-run has unbounded latency and may fail).  Its scratch lives
 * in a static 16 MiB device array inside the library (held by every GPU that
 * loads it, until exit); a dataset whose scratch would not fit -- for the
 * float-float shapes beyond about 2e8 events with 6 gradient slots, 1.4e8
 * with 12; for the generic kernel about 5e8 and 3e8 -- is rejected with
 * RF_E_INVALID and a message giving the limit
 * (rf_nll_grad_noalloc_max_events).
 *   d_cols : n_obs DEVICE column pointers (host array of pointers), dtype per
 *            column (NULL = all RF_F64), n_events events each.
 *   d_theta: DEVICE n_free parameters; d_out: DEVICE 1 + n_free doubles (NLL,
 *            gradient); d_flags: DEVICE int32, events with pdf <= 0 / not
 *            finite (+2^30 when theta is outside a pdf's domain).
 * Asynchronous on `stream`.  All calls on a device share the array, so calls
 * that overlap on the GPU race and must be serialised by the caller.  The
 * first call on each device looks the array up (cudaGetSymbolAddress) with
 * that device current; make it before any stream capture. */
rf_status rf_nll_grad_noalloc(const rf_model* m, const void* const* d_cols, const int32_t* dtype, int64_t n_events,
                              const double* d_theta, double* d_out, int32_t* d_flags, void* stream);
/* The largest n_events that rf_nll_grad_noalloc accepts for model m (its
 * scratch grows with the number of 4096-event chunks and with the model's
 * gradient slots); larger datasets are rejected.  Host only: touches no
 * device. */
rf_status rf_nll_grad_noalloc_max_events(const rf_model* m, int64_t* max_events);

/* -------------------------------------------------------------- messages */

const char* rf_last_error(void);
const char* rf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RF_H */

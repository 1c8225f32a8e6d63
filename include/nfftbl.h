/*
 * nfftbl -- nonequispaced fast Fourier transforms for bandlimited functions
 * on one GB300 (sm_103a).
 *
 * The library evaluates the NFFT-like procedure for bandlimited functions of
 * Kircheis & Potts (Algorithm 4.2, matrix form f = Psi F D_psihat fhat of
 * Eq. 4.11), its adjoint D_psihat F^H Psi^T, and the classical NFFT
 * (Algorithm 2.1, A ~ B F D of Eqs. 2.2-2.6) on the same inputs.
 *
 * Problem (Section 1, Eq. 1.1 and the statement opening Section 4): given
 * samples fhat(k), k in I_M = [-M/2, M/2)^d, of the Fourier transform of a
 * bandlimited f, approximate f(x_j) at nodes x_j in [-1/2, 1/2)^d, d = 1..3.
 *
 * Storage conventions (the paper leaves them open):
 *   - complex values are interleaved (re, im): complex64 (float2) for
 *     single-precision plans, complex128 (double2) for double-precision plans;
 *   - fhat is centred and row-major with dimension 0 slowest: element k sits
 *     at sum_t (k_t + M_t/2) * prod_{s>t} M_s; a batch of B vectors is
 *     B contiguous blocks of prod_t M_t elements;
 *   - nodes x are N x d row-major, float (single plans) or double (double
 *     plans), each coordinate in [-1/2, 1/2);
 *   - f (length N per batch entry) is in the caller's node order; a batch is
 *     B contiguous blocks of N elements.
 *
 * Ownership: every pointer argument named *_dev is caller-owned device memory
 * (for example a torch tensor's storage) that must stay valid until the call's
 * work on the plan's stream has finished; the library never frees it.  The
 * plan owns its own buffers (window factors, grid, sorted nodes, tile
 * tables, scratch) and releases them in nfftbl_destroy.
 *
 * Errors: every entry point returns an nfftbl_status; NFFTBL_OK is 0.  On any
 * other status the plan keeps its previous valid state and
 * nfftbl_last_error(plan) describes the failure.  No C++ exception crosses
 * this interface.  Work is enqueued asynchronously on the plan's stream;
 * nfftbl_set_nodes is the only call that synchronises (it reads back a
 * domain-check flag and the work-list size).
 */
#ifndef NFFTBL_H
#define NFFTBL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nfftbl_plan_s* nfftbl_plan_t;

typedef enum {
    NFFTBL_OK = 0,
    NFFTBL_EINVAL = 1,        /* invalid argument (sizes, NULL pointers)          */
    NFFTBL_EDOMAIN = 2,       /* a node outside [-1/2, 1/2)^d or NaN              */
    NFFTBL_EUNSUPPORTED = 3,  /* valid in the paper but not built (e.g. L not 2^p) */
    NFFTBL_ENOMEM = 4,        /* device allocation failed                         */
    NFFTBL_ECUDA = 5,         /* a CUDA runtime/driver call failed                */
    NFFTBL_ESTATE = 6,        /* call order violated (e.g. forward before nodes)  */
    NFFTBL_ETIMEOUT = 7,      /* a bounded device-side wait gave up               */
    NFFTBL_EINTERNAL = 8      /* internal consistency check failed                */
} nfftbl_status;

/* Window functions of the class Phi_{m,L} (Section 3, Remark 3.1). */
typedef enum {
    NFFTBL_WIN_SINH = 0,   /* Eq. 3.4: sinh(beta sqrt(1-(Lx/m)^2)) / sinh(beta)          */
    NFFTBL_WIN_CKB = 1,    /* continuous Kaiser-Bessel: (I0(beta sqrt(.)) - 1)/(I0(beta) - 1) */
    NFFTBL_WIN_TABLE = 2   /* caller-supplied table on u = |Lx|/m in [0,1] (learned window) */
} nfftbl_window;

typedef enum {
    NFFTBL_F64 = 0,        /* double everywhere                                           */
    NFFTBL_F32 = 1,        /* float data and arithmetic; FP64-derived weights and twiddles */
    NFFTBL_F32_COMP = 2    /* as F32 with compensated (Neumaier) accumulation of tap rows  */
} nfftbl_precision;

typedef enum {
    NFFTBL_SHANNON = 0,    /* Algorithm 4.2: kernel psi = sinc(L pi x) phi(x), zero extension */
    NFFTBL_CLASSIC = 1     /* Algorithm 2.1: periodized window phi_m                            */
} nfftbl_method;

typedef struct {
    int precision;          /* nfftbl_precision; default NFFTBL_F32                       */
    int method;             /* nfftbl_method; default NFFTBL_SHANNON                      */
    double beta;            /* window shape; <= 0 selects the default: pi m (1 - 1/sigma)
                               for SHANNON, 2 pi m (1 - 1/(2 sigma)) for CLASSIC            */
    int batch;              /* B >= 1 transforms sharing the nodes; default 1             */
    const double* table;    /* host pointer, NFFTBL_WIN_TABLE only: values g(u_i) at
                               u_i = i/(table_len-1), i = 0..table_len-1, copied by the plan */
    int table_len;          /* >= 3 for NFFTBL_WIN_TABLE                                  */
    int tile[3];            /* node-binning tile shape in grid cells; 0 = default         */
    int nodes_per_item;     /* nodes per (tile, chunk) work item, <= 2047; 0 = default 1024 */
    int factors;            /* step 0b of Algorithm 4.2 in tensor-product form: 1 keeps the
                               d x 2m window factors of every node, computed once by
                               nfftbl_set_nodes (N * d * 2m values in the plan precision,
                               rows padded to 4); 0 (default) evaluates them in every
                               transform, which is faster on GB300 for the sinh window  */
    int precorrect;         /* 1 (default): D_psihat = diag(1/(|I_L| psi_hat(k))) of Eq. 4.9
                               (D of Eq. 2.2); 0: D = I, the approximation of Section 5
                               that uses |I_L| psi_hat(k) ~ 1 (an ablation)             */
    int weights;            /* tap weights psi(x_j - l/L) of the spreading (transposed
                               step 3) in FP32 plans with m <= 8: 0 (default) the window's
                               closed form per tap; 1: one polynomial per tap in the node's
                               offset, fitted in FP64 when the plan is made and kept only
                               if it is accurate to 3e-7 of the largest weight (FP32
                               evaluation included).  The interpolation and the node
                               derivative always use the closed form                    */
} nfftbl_opts;

/* Fill *opts with the defaults listed above. */
void nfftbl_default_opts(nfftbl_opts* opts);

/*
 * Create a plan (Algorithm 4.2 step 0a / Algorithm 2.1 step 0a).
 *   out    : receives the plan handle (NULL on failure);
 *   d      : dimension, 1..3;
 *   M      : host array of d even band sizes M_t >= 2 (|I_M| = prod M_t);
 *   sigma  : oversampling factor >= 1; L_t = 2 ceil(ceil(sigma M_t)/2)
 *            (M_sigma of Algorithm 2.1; L = M(1+lambda) in Algorithm 4.2);
 *   m      : truncation parameter, window support [-m/L, m/L];
 *   window : nfftbl_window;
 *   opts   : NULL for defaults.
 * Computes on the device, in FP64, the window transform psi_hat (phi_hat for
 * CLASSIC) at k in I_{M_t} per dimension by Gauss-Legendre quadrature, and the
 * diagonal D_psihat = diag(1/(|I_L| psi_hat(k))) of Eq. 4.9 (D of Eq. 2.2) in
 * tensor-product form.  Runs on the legacy default stream and synchronises.
 * Errors: EINVAL (d, M odd or < 2, sigma < 1, m < 1, 2m >= L_t, batch < 1,
 * bad table or tile, beta <= 0 after defaults), EUNSUPPORTED (L_t not of
 * the form 2^a 3^b 5^c in [16, 4096] -- the FFT's radices --, m outside
 * 2..12, prod L_t > 2^31, a box of tile plus halo beyond shared memory:
 * with the smallest tiles this limits d = 3 to m <= 8 in FP64 and m <= 9 in
 * FP32),
 * ENOMEM, ECUDA.  Tiles are the largest power of two (up to 64 / 32^2 / 8^3
 * for d = 1 / 2 / 3) dividing L_t.  The message of a
 * failed call is available from nfftbl_plan_error().
 */
nfftbl_status nfftbl_plan(nfftbl_plan_t* out, int d, const int* M, double sigma, int m,
                          int window, const nfftbl_opts* opts);

/* Enqueue all later work of this plan on cuda_stream (a cudaStream_t; NULL =
 * legacy default stream).  Never fails for a valid plan. */
nfftbl_status nfftbl_set_stream(nfftbl_plan_t plan, void* cuda_stream);

/*
 * Set the nodes x_j (Algorithm 4.2 inputs; index set J_{L,m}(x) of Eq. 4.8).
 *   N     : number of nodes, 0 <= N < 2^31;
 *   x_dev : N x d device array (float for F32/F32_COMP plans, double for F64),
 *           row-major; may be freed by the caller once this call returns.
 * Bins the nodes into grid tiles: cell i_t = floor(L_t x_t) + L_t/2, tile and
 * in-tile cell key, stable order by (key, j), tile offsets and the work list.
 * Synchronises the stream.  Errors: EINVAL, EDOMAIN (a coordinate outside
 * [-1/2, 1/2) or NaN; the plan then has no nodes), ENOMEM, ECUDA.
 */
nfftbl_status nfftbl_set_nodes(nfftbl_plan_t plan, int64_t N, const void* x_dev);

/*
 * Forward transform f = Psi F D_psihat fhat (Eq. 4.11; Algorithm 4.2 steps
 * 1-3), or f = B F D fhat for CLASSIC (Algorithm 2.1).
 *   fhat_dev : B x prod(M_t) complex input (centred, row-major);
 *   f_dev    : B x N complex output in the caller's node order.
 * The plan's grid keeps the equispaced values vartheta_l (Eq. 4.7) until the
 * next transform.  Asynchronous: errors: ESTATE (no nodes set), EINVAL
 * (NULL), ECUDA (launch failure).  Device-side failures (a bounded wait on a
 * tile copy that gave up) are reported by the next nfftbl_sync.
 */
nfftbl_status nfftbl_forward(nfftbl_plan_t plan, const void* fhat_dev, void* f_dev);

/*
 * Adjoint transform fhat = D_psihat F^H Psi^T f (the transpose of Eq. 4.11;
 * the paper does not state it), or D F^H B^T f for CLASSIC.
 *   f_dev    : B x N complex input in the caller's node order;
 *   fhat_dev : B x prod(M_t) complex output (centred, row-major).
 * The grid is overwritten.  Errors as for nfftbl_forward.
 */
nfftbl_status nfftbl_adjoint(nfftbl_plan_t plan, const void* f_dev, void* fhat_dev);

/*
 * Node gradient: gradx[j, t] = sum_b Re(conj(gradf[b, j]) * d f_{b,j} / d x_{j,t})
 * for the forward map of this plan (not in the paper; the derivative of the
 * short sums of Algorithm 4.2 step 3 with respect to the node).
 *   fhat_dev  : B x prod(M_t) complex (the forward input);
 *   gradf_dev : B x N complex (gradient with respect to f);
 *   gradx_dev : N x d real output (float or double, the plan's precision).
 * Recomputes the grid from fhat.  Errors as for nfftbl_forward.
 */
nfftbl_status nfftbl_node_grad(nfftbl_plan_t plan, const void* fhat_dev, const void* gradf_dev,
                               void* gradx_dev);

/*
 * Forward and adjoint transforms with HOST input and output (same maps as
 * nfftbl_forward / nfftbl_adjoint: Eq. 4.11 of Algorithm 4.2 and its
 * transpose; Algorithm 2.1 for CLASSIC).
 *   fhat_host : B x prod(M_t) complex, centred row-major (as fhat_dev);
 *   f_host    : B x N complex in the caller's node order (as f_dev).
 * The input is copied into a plan-owned device staging buffer on the plan's
 * upload stream, the transform runs on the plan stream, and the output is
 * copied back on the plan's download stream; events order each staging
 * buffer between its copies and the transform that uses it, so consecutive
 * calls overlap: the upload of an adjoint's input runs during the preceding
 * forward transform, the download of a forward's output during the
 * following adjoint.  Asynchronous: the outputs are in host memory after
 * nfftbl_sync, or when work enqueued on the plan stream after nfftbl_join
 * has completed.  The caller keeps the host buffers alive and unmodified
 * (inputs) or unread (outputs) until then.  Page-locked host memory gives
 * asynchronous copies; pageable memory works, with the copies staged
 * synchronously by the CUDA runtime.  Errors as for nfftbl_forward, plus
 * ENOMEM for the staging buffers (allocated on first use, kept until the
 * plan is destroyed).
 */
nfftbl_status nfftbl_forward_host(nfftbl_plan_t plan, const void* fhat_host, void* f_host);
nfftbl_status nfftbl_adjoint_host(nfftbl_plan_t plan, const void* f_host, void* fhat_host);

/* Make later work on the plan stream wait for the downloads issued by the
 * host-buffer calls so far (no host blocking).  Never fails for a valid plan
 * whose CUDA context is healthy. */
nfftbl_status nfftbl_join(nfftbl_plan_t plan);

/* Wait for the plan's stream (and the upload and download streams of the
 * host-buffer calls) and report device-side failures of the work
 * enqueued so far: ETIMEOUT if a bounded wait gave up (results invalid),
 * EINTERNAL for another device error word; the word is cleared. */
nfftbl_status nfftbl_sync(nfftbl_plan_t plan);

/* Limit of the plan's bounded device-side waits (the interpolation and
 * node-derivative kernels' waits for a TMA tile copy), in nanoseconds of the
 * GPU's global timer: limit_ns in [1, 6e10]; 0 restores the default of 2 s.
 * A wait that runs out abandons the transform (its outputs are invalid),
 * lets its copy in flight land, sets the plan's device error word and
 * returns, so that the CUDA context stays usable; the next nfftbl_sync
 * reports ETIMEOUT and clears the word.
 * stall_next != 0 arms a test of that path: in the next interpolation
 * launch the tile waits are armed but no copy is issued, so nothing can
 * complete them and every wait runs out after limit_ns (a failure made on
 * purpose, without faulting the device).  Not in the paper: a safety
 * device of this implementation.  Errors: EINVAL (NULL plan, limit out of
 * range). */
nfftbl_status nfftbl_set_wait_limit(nfftbl_plan_t plan, int64_t limit_ns, int stall_next);

/* Release the plan and all of its device memory.  NULL is accepted.  The
 * handle must not be used again. */
nfftbl_status nfftbl_destroy(nfftbl_plan_t plan);

/* Text of the last error on this plan ("" if none; a static message for a NULL
 * plan).  Valid until the next call on the plan. */
const char* nfftbl_last_error(nfftbl_plan_t plan);

/* Text of the last failure in this thread of a call that has no plan to hold
 * it: nfftbl_plan (the plan handle is NULL then) and nfftbl_grid_noalloc. */
const char* nfftbl_plan_error(void);

/* ---------------------------------------------------------------------------
 * Introspection, for tests and benchmarks.  All copy to caller-owned HOST
 * memory and synchronise the plan's stream.
 * ------------------------------------------------------------------------ */

typedef struct {
    int d, M[3], L[3], m, precision, method, window, batch;
    double beta;
    int tile[3];
    int64_t n_nodes;
    int64_t n_tiles;
    int64_t n_work;         /* work items (tile, chunk) after set_nodes              */
    int key_bits;           /* bits of the binning key                               */
    int poly_weights;       /* 1: the short sums use the per-tap weight polynomials     */
    double poly_err;        /* their largest error relative to the largest weight (0 if
                               no fit was made)                                          */
} nfftbl_info;

/* The plan's parameters (after defaults: L_t, beta, tile extents) and, once
 * nodes are set, the binning sizes, into caller-owned host memory.  Errors:
 * EINVAL (NULL plan or info). */
nfftbl_status nfftbl_get_info(nfftbl_plan_t plan, nfftbl_info* info);

/* Precorrection factors of dimension t: d_t(k) = 1/(L_t psi_hat_t(k)),
 * k in I_{M_t} centred (M_t doubles), so that D = prod_t d_t (Eq. 4.9). */
nfftbl_status nfftbl_get_factors(nfftbl_plan_t plan, int t, double* host_out);

/* Binning results after set_nodes: keys (N uint32, sorted order), perm (N
 * uint32, original index of each sorted node), tile_off (n_tiles+1 uint32).
 * Any pointer may be NULL to skip it. */
nfftbl_status nfftbl_get_binning(nfftbl_plan_t plan, uint32_t* keys, uint32_t* perm,
                                 uint32_t* tile_off);

/* Copy the current grid (B x prod(L_t) complex, centred) into host memory. */
nfftbl_status nfftbl_get_grid(nfftbl_plan_t plan, void* host_out);

/* Device address of the plan's grid (B x prod(L_t) complex, centred) so that
 * a caller may run step 3 (or its adjoint) on a grid it filled itself. */
nfftbl_status nfftbl_grid_ptr(nfftbl_plan_t plan, void** grid_dev);

/* The window transform at arbitrary real frequencies v (Eq. 4.2 for the
 * Shannon method: psi_hat(v) = int sinc(L pi x) phi(x) e^{-2 pi i v x} dx;
 * phi_hat(v) for CLASSIC), dimension t, in FP64 by the plan's own device
 * quadrature (the rule of step 0a).  v_dev, out_dev: device arrays of n
 * doubles.  Used for approximations at non-integer frequencies (Section 5,
 * Fig. 5.1: the classical approximation divides by L phi_hat(v)).
 * Asynchronous on the plan's stream.  Errors: EINVAL (t, n, NULL). */
nfftbl_status nfftbl_window_transform(nfftbl_plan_t plan, int t, const double* v_dev, int n, double* out_dev);

/*
 * Step 3 alone (Algorithm 4.2 step 3 / Algorithm 2.1 step 3): f = Psi grid
 * from the plan's current grid, and its transpose grid = Psi^T f (the grid is
 * cleared first).  For experiments that supply equispaced samples directly,
 * such as the exponential approximations of Eqs. 5.1-5.2.
 */
nfftbl_status nfftbl_interp_grid(nfftbl_plan_t plan, void* f_dev);
nfftbl_status nfftbl_spread_grid(nfftbl_plan_t plan, const void* f_dev);

/* Number of this library's kernels launched on the plan so far (all calls). */
int64_t nfftbl_kernel_launches(nfftbl_plan_t plan);

/* Kernel classes for the per-kernel timers below. */
typedef enum {
    NFFTBL_K_FFT = 0,       /* FFT passes (steps 1-2 and their adjoint)     */
    NFFTBL_K_INTERP = 1,    /* short sums, step 3                           */
    NFFTBL_K_SPREAD = 2,    /* transposed short sums                        */
    NFFTBL_K_GRAD = 3,      /* node derivative                              */
    NFFTBL_K_BIN = 4,       /* binning (keys, sort, offsets)                */
    NFFTBL_K_FLUSH = 5,     /* ordered flush of the spread boxes to the grid */
    NFFTBL_K_COUNT = 6
} nfftbl_kernel_class;

/* enable != 0: record a CUDA event pair on the plan's stream around every
 * later kernel launch of this plan (adds two event records per launch);
 * enable == 0: stop recording.  Either way the accumulated times are reset. */
nfftbl_status nfftbl_kernel_timing(nfftbl_plan_t plan, int enable);

/* Synchronise the recorded events and return, per kernel class, the summed
 * device time in milliseconds (ms_out) and the number of launches
 * (count_out), each an array of NFFTBL_K_COUNT entries (host memory).  The
 * accumulators are reset afterwards. */
nfftbl_status nfftbl_kernel_times(nfftbl_plan_t plan, double* ms_out, int64_t* count_out);

/* ---------------------------------------------------------------------------
 * Learned window (tabulated window trained on the transform's own error).
 *
 * The window class Phi_{m,L} of Section 3 admits windows other than the two
 * of Remark 3.1; these calls let a tabulated window phi(u), u = |Lx|/m, be
 * produced by a small MLP and trained on the device:
 *   phi_theta(u) = (1 - u^2) exp(g(u^2) - g(0)),
 *   g(s) = W3 tanh(W2 tanh(W1 s + b1) + b2) + b3   (1 -> 64 -> 64 -> 1).
 * Parameter layout (float): W1[64], b1[64], W2[64][64] (out x in), b2[64],
 * W3[64], b3[1] (nfftbl_mlp_param_count(64) values).
 * ------------------------------------------------------------------------ */

/* Replace the plan's table (plan made with NFFTBL_WIN_TABLE) by table_len
 * doubles in device memory and recompute psi_hat and D_psihat (Alg. 4.2
 * step 0a) on the plan's stream.  No allocation.  Errors: EINVAL (length
 * differs from the plan's), ESTATE (not a table window), ECUDA. */
nfftbl_status nfftbl_set_window_table(nfftbl_plan_t plan, const double* table_dev, int table_len);

/* Loss of the transform against targets and its gradient with respect to
 * the window table (FP32 Shannon plans with a table window, d <= 2):
 *   E = ||f - y||^2 / ||y||^2,   f = Psi F D_psihat fhat (Eq. 4.11),
 * dE/dv through both the short-sum weights and the precorrection (the
 * quadrature that forms psi_hat from the table).
 *   fhat_dev       : B x prod(M_t) complex64;   y_dev : B x N complex64 (caller order);
 *   grad_table_dev : table_len doubles (overwritten);
 *   loss_dev       : 3 doubles (overwritten): E, ||f - y||^2, ||y||^2.
 * Overwrites the plan's grid.  Asynchronous.  Errors: ESTATE (no nodes, not a
 * Shannon table plan), EUNSUPPORTED (FP64 or d = 3), ENOMEM, ECUDA. */
nfftbl_status nfftbl_window_loss_grad(nfftbl_plan_t plan, const void* fhat_dev, const void* y_dev,
                                      double* grad_table_dev, double* loss_dev);

/* Evaluate the MLP at u_i = i/(table_len-1) and write the window table
 * (doubles, device).  act_dev receives the activations the backward pass
 * needs: table_len * (2*hidden + 1) floats.  FP32 arithmetic.  hidden must be
 * 64 (EUNSUPPORTED otherwise). */
nfftbl_status nfftbl_mlp_table(const float* params_dev, int hidden, int table_len, double* table_dev,
                               float* act_dev, void* cuda_stream);

/* Gradient of the loss with respect to the MLP parameters from its gradient
 * with respect to the table (chain rule through v_i = (1-u_i^2) exp(g_i - g_0)
 * and back-propagation through the MLP; the two 64-wide matrix products run
 * on the tensor cores in BF16 with FP32 accumulation).  scratch_dev: at least
 * nfftbl_mlp_scratch_floats(hidden, table_len) floats; grad_params_dev:
 * nfftbl_mlp_param_count(hidden) floats (overwritten). */
nfftbl_status nfftbl_mlp_backward(const float* params_dev, int hidden, int table_len, const float* act_dev,
                                  const double* table_dev, const double* grad_table_dev, float* scratch_dev,
                                  float* grad_params_dev, void* cuda_stream);

/* Parameter count of the MLP (-1 if hidden != 64) and scratch size (floats)
 * of nfftbl_mlp_backward (-1 if unsupported). */
int64_t nfftbl_mlp_param_count(int hidden);
int64_t nfftbl_mlp_scratch_floats(int hidden, int table_len);

/* One Adam step (bias-corrected, step >= 1) on count parameters, all device
 * arrays of floats: params -= lr * mhat / (sqrt(vhat) + eps). */
nfftbl_status nfftbl_adam_step(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int count,
                               int step, float lr, float beta1, float beta2, float eps, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Allocation-free equispaced samples.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: code running under another framework's memory
 * pool or allocator hooks (where a library's own device allocations are not
 * allowed or not visible to the owner of the memory), or hosts that only hand
 * out buffers they allocated themselves.  nfftbl_plan allocates (window
 * factors, grid, scratch), so such callers cannot use a plan; this call needs
 * none.
 *
 * It computes what nfftbl_forward computes before its short sums: the
 * precorrected, zero-padded, oversampled inverse FFT of fhat, i.e. the
 * equispaced samples the short sums read, for the Shannon method with the
 * sinh window, in FP32:
 *   d, M, sigma, m, beta, batch : as for nfftbl_plan (beta <= 0: default
 *                                 pi m (1 - 1/sigma)); batch B >= 1;
 *   fhat_dev  : B x prod(M_t) complex64 input (centred, row-major), caller-owned;
 *   grid_dev  : B x prod(L_t) complex64 output (centred, row-major), caller-owned;
 *   cuda_stream : cudaStream_t the work is enqueued on (NULL = legacy stream).
 * The result equals the grid a plan with the same parameters holds after
 * nfftbl_forward.  L_t = 2^a 3^b 5^c in [16, 4096], as for nfftbl_plan.
 *
 * It allocates nothing: the window factors, twiddles and intermediate FFT
 * passes live in one fixed device array of 16 MiB inside the library, which
 * every GPU that loads the library holds until the process exits.  Problems
 * whose factors, twiddles and intermediates need more than 16 MiB
 * (d = 2: about B * M_0 * L_1 * 8 bytes; d = 3: B * M_0 * L_2 * (M_1 + L_1) * 8
 * bytes) are rejected with NFFTBL_EINVAL and a message naming the size.
 * The first call on a device sets that device up, with the device current:
 * it looks up the device's address of the array and copies the quadrature
 * rule of the window factors to the device (a synchronous copy); make the
 * first call on each device before any stream capture.  Later calls only
 * launch kernels.  A call whose parameters (d, M, L, m, beta) equal the
 * previous call's on the same device reuses the window factors that call
 * left in the array instead of repeating their quadrature.
 * Every call shares the one array and leaves its contents behind: calls
 * whose work overlaps on the GPU (different streams, or different threads
 * without ordering) race on it, so serialise them.  The device address is
 * looked up once per process and device: calls after cudaDeviceReset (or any
 * other re-creation of the device's primary context) are not supported.
 * Asynchronous; errors: EINVAL, EUNSUPPORTED (as for nfftbl_plan), ECUDA.
 * The message of a failed call is available from nfftbl_plan_error().
 */
nfftbl_status nfftbl_grid_noalloc(int d, const int* M, double sigma, int m, double beta, int batch,
                                  const void* fhat_dev, void* grid_dev, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* NFFTBL_H */

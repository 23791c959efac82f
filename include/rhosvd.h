/*
 * rhosvd.h -- C ABI of the GB300 (sm_103a) RHOSVD library.
 *
 * Reduced HOSVD canonical-to-Tucker (C2T) rank reduction of a d = 3 canonical tensor
 *   A = sum_{nu=1}^R xi_nu u_nu^(1) (x) u_nu^(2) (x) u_nu^(3)          (Sec. 2.1, eq. can_A3)
 * into the orthogonal Tucker tensor
 *   A0 = beta x_1 Z^(1) x_2 Z^(2) x_3 Z^(3),                            (Def. 2.2, eq. RHOSVD)
 * where Z^(l) (n_l x r_l) spans the dominant left singular subspace of the normalised side
 * matrix U^(l) (eq. SVD_Ul, eq. svdr) and the core is the Khatri-Rao contraction
 *   beta(i,j,m) = sum_nu xi_nu V^(1)(i,nu) V^(2)(j,nu) V^(3)(m,nu),  V^(l) = Z^(l)T U^(l)
 * (Prop. 2.2).  Plus the canonical Hadamard product and sum whose rank growth RHOSVD cuts
 * back (Sec. 3 eq. rho_ten; Lemma 4.2; Sec. 4.3).
 *
 * Conventions for every entry point:
 *   - Pointers named in a struct are DEVICE pointers unless stated otherwise; the caller
 *     owns every buffer (inputs, outputs, workspace).  Inputs are never written.
 *   - Matrices are column-major; U^(l) is n_l x R with leading dimension ld_l >= n_l.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 *     Host-side argument errors are returned immediately; results and device-side
 *     status land in `rhosvd_info` (device memory) and are valid after a stream sync.
 *   - The library never aborts, never throws, never prints and never allocates memory in
 *     rhosvd_c2t / rhosvd_cp_hadamard / rhosvd_cp_sum.
 *   - Return value: RHOSVD_OK or a negative RHOSVD_ERR_* code.
 */
#ifndef RHOSVD_H
#define RHOSVD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RHOSVD_OK 0
#define RHOSVD_ERR_INVALID_ARG (-1)     /* bad sizes, NULL pointers, unsupported options    */
#define RHOSVD_ERR_RANK_OVERFLOW (-2)   /* device: some r_l > r_max (needed rank in info)   */
#define RHOSVD_ERR_NOT_CONVERGED (-3)   /* device: a small factorisation broke down          */
#define RHOSVD_ERR_NONFINITE (-4)       /* device: Inf/NaN in factors or weights             */
#define RHOSVD_ERR_SKETCH (-5)          /* device: sketch residual alone exceeds eps         */
#define RHOSVD_ERR_CUDA (-6)            /* a CUDA launch/runtime call failed                 */
#define RHOSVD_ERR_WORKSPACE (-7)       /* workspace NULL or smaller than required          */
#define RHOSVD_ERR_SCRATCH_LIMIT (-8)   /* rhosvd_c2t_noalloc: problem exceeds the static scratch */
#define RHOSVD_ERR_TIMEOUT (-9)         /* device: a bounded wait inside a kernel gave up      */

#define RHOSVD_PLAIN_FP64 0             /* every step in FP64 on the CUDA cores              */
#define RHOSVD_MIXED 1                  /* the large contractions (range sketch, Grams,
                                           projection, Ritz vectors, residual, core) on the
                                           tcgen05 tensor cores with exact digit planes held as
                                           BF16 (seven 7-bit digits for the FP64-class products,
                                           five for the range sketch when every rank is chosen
                                           by eps and eps >= 1.5e-9 sqrt(max n), four 8-bit
                                           digits for the core) and FP32 accumulation read back
                                           into FP64 (about 2^-40 of sum|a||b| for the core);
                                           the small factorisations stay FP64                  */

#define RHOSVD_K_MAX 256                /* largest subspace width k handled on the device    */

/* A d = 3 canonical tensor (Sec. 2.1, eq. can_A3).  Factor columns need not be
 * normalised: the library normalises them and folds the norms into the weights. */
typedef struct rhosvd_cp {
    int n[3];               /* mode sizes n_l >= 1                                        */
    int R;                  /* canonical rank R >= 0                                      */
    const double* U[3];     /* U^(l): n_l x R, column-major, leading dimension ld[l]      */
    int ld[3];              /* ld[l] >= n[l]                                              */
    const double* xi;       /* weights xi_nu, length R (may be signed)                    */
} rhosvd_cp;

typedef struct rhosvd_opts {
    double eps;             /* relative Frobenius threshold per mode: r_l is the smallest r
                               with sum_{k>r} sigma_{l,k}^2 <= eps^2 sum_k sigma_{l,k}^2
                               (the epsilon-threshold of Thm. 2.3); energy at or below the
                               FP64 resolution (n_l u)^2 sum_k sigma_{l,k}^2 counts as zero,
                               so eps = 0 keeps every direction FP64 resolves             */
    int ranks[3];           /* > 0: fixed r_l = min(ranks[l], rank bound); 0: use eps     */
    int r_max;              /* capacity of the outputs; 1 <= r_max <= RHOSVD_K_MAX        */
    int oversample;         /* sketch columns beyond r_max (k = r_max + oversample)       */
    int precision;          /* RHOSVD_PLAIN_FP64 or RHOSVD_MIXED                          */
    int deflate;            /* width of the second range sketch, taken on the residual of the
                               first basis (Y2 = (I - Q Q^T) U Omega2) and appended to it:
                               0 = the default (16), < 0 = none, 1..64 = that width.  It
                               finds the directions whose singular values sit near sqrt(u)
                               of the largest, which a Gram-based orthonormalisation of a
                               single sketch cannot resolve (needed for eps near 1e-7)   */
    unsigned long long seed;/* seed of the counter-based sketch generator                 */
    int out_fp32;           /* 0: Z^(l) and beta written as double; 1: written as float
                               (FP32, each entry the FP64 result rounded once to nearest;
                               the capacities below stay counted in entries).  sigma, V,
                               xi_out and info keep their FP64 types.  Accepted by
                               rhosvd_c2t, _noalloc, _batched, _hadamard, _start and _als;
                               rhosvd_cp_horner, whose steps read their own Tucker
                               tensors back, rejects it (INVALID_ARG)                     */
} rhosvd_opts;

/* Device-written result record (one per call).  Valid after the stream is synchronised. */
typedef struct rhosvd_info {
    int status;             /* RHOSVD_OK or a device-side RHOSVD_ERR_* code              */
    int r[3];               /* Tucker ranks r_l actually stored                           */
    int r_needed[3];        /* rank the eps rule asked for (== r unless RANK_OVERFLOW)     */
    int k[3];               /* width of the orthonormal basis Q^(l) after rank revealing   */
    int kept;               /* canonical terms kept after dropping zero terms             */
    int direct[3];          /* 1 if mode l used the exact n_l x n_l Gram (no sketch)       */
    double xi_norm;         /* ||xi'|| of the normalised weights (Thm. 2.3)              */
    double total[3];        /* ||U^(l) normalised||_F^2                                   */
    double resid[3];        /* ||U - Z_hi V_hi||_F^2: energy outside the leading directions
                               computed as rank candidates (<= eps^2 total unless SKETCH)  */
    double tail[3];         /* tau_l = ||U^(l) - Z^(l) V^(l)||_F measured directly, the
                               per-mode truncation error of Thm. 2.3                       */
} rhosvd_info;

/* Outputs of rhosvd_c2t (all device memory, caller-allocated). */
typedef struct rhosvd_tucker {
    void* Z[3];             /* Z^(l): n_l x r_max, ld n_l; columns >= r_l are zero; double
                               entries, or float with opts->out_fp32                      */
    void* beta;             /* capacity r_max^3 entries (double, or float with out_fp32);
                               the r1 x r2 x r3 core packed densely, beta[i + r1 (j + r2 m)] */
    double* sigma[3];       /* capacity RHOSVD_K_MAX each: sigma_{l,1..k_l}, descending,
                               zero beyond k_l                                            */
    double* V[3];           /* optional (NULL = not returned): r_max x R, ld r_max; rows
                               < r_l hold V^(l) = Z^(l)T U^(l)_normalised = D_{l,0} V_0^T,
                               the mixed Tucker-canonical core factors (Prop. 2.2)        */
    double* xi_out;         /* optional (NULL = not returned): the R normalised weights   */
    rhosvd_info* info;      /* required                                                  */
} rhosvd_tucker;

/* Library version (major * 10000 + minor * 100 + patch). */
int rhosvd_version(void);

/* Message for a status code (static storage). */
const char* rhosvd_strerror(int code);

/* Bytes of device workspace rhosvd_c2t needs for this tensor and these options, or 0 if
 * the arguments are invalid.  Depends only on sizes and options. */
size_t rhosvd_c2t_workspace_size(const rhosvd_cp* cp, const rhosvd_opts* opts);

/* Width of the subspace searched in mode l (k_l before rank revealing); -1 on bad args. */
int rhosvd_subspace_width(const rhosvd_cp* cp, const rhosvd_opts* opts, int mode);

/*
 * RHOSVD canonical-to-Tucker transform (Def. 2.2, Prop. 2.2, Thm. 2.3).
 * Steps, all on the device: normalise the canonical vectors (Sec. 2.1); per mode find an
 * orthonormal basis Q of the range of U^(l) (the exact identity when n_l <= k, else a
 * randomised range sketch U^(l) Omega with Rademacher Omega); project B = Q^T U^(l);
 * eigen-decompose B B^T to get the singular values and left singular vectors inside
 * span(Q) (eq. SVD_Ul restricted to Q); choose r_l by the eps rule; write
 * Z^(l) = Q W_r, V^(l) = W_r^T B and the Khatri-Rao core beta.
 * workspace: device memory of at least rhosvd_c2t_workspace_size() bytes, 256-byte aligned.
 * Errors: RHOSVD_ERR_INVALID_ARG, RHOSVD_ERR_WORKSPACE, RHOSVD_ERR_CUDA (returned);
 *         RANK_OVERFLOW, NOT_CONVERGED, NONFINITE, SKETCH (in info->status).
 */
int rhosvd_c2t(const rhosvd_cp* cp, const rhosvd_opts* opts, const rhosvd_tucker* out,
               void* workspace, size_t workspace_bytes, void* stream);

/*
 * RHOSVD followed by ALS sweeps toward the best rank-r Tucker approximation (Sec. 2.2, the ALS
 * step after Def. 2.2, eq. can_A_Tuck_als).  The ranks r_l are the RHOSVD's (eps rule or fixed).
 * One sweep updates the modes 0, 1, 2 in turn: with the other two factors fixed, the contraction
 * of the canonical tensor with them has the mode-l unfolding U~_l diag(xi') (V_m2 (.) V_m1)^T
 * (V_m = Z_m^T U~_m), and Z_l becomes its r_l leading left singular vectors.  The step is taken
 * inside the RHOSVD's orthonormal basis Q_l of the side matrix (the sketch range, or the identity
 * for a direct mode): C_l = (Q_l^T U~_l) diag(xi') (V_m2 (.) V_m1)^T, W_l = the r_l leading
 * eigenvectors of C_l C_l^T, Z_l = Q_l W_l.  Each step cannot lower the captured energy
 * ||beta||^2, so the Tucker error ||A||^2 - ||beta||^2 never grows.  All ALS products run in FP64
 * on the CUDA cores (the RHOSVD part follows opts->precision).
 *   sweeps     0 .. RHOSVD_ALS_MAX_SWEEPS (0 = plain rhosvd_c2t)
 *   out        as rhosvd_c2t: Z, beta and V are the refined ones; sigma and info (tail, resid)
 *              describe the RHOSVD start
 *   energy     host array of 6 sweeps doubles or NULL: for step s = 3 sweep + l, energy[2 s] is
 *              ||beta||^2 before and energy[2 s + 1] after the mode-l update (the call then
 *              synchronises `stream`; with NULL it stays asynchronous)
 *   workspace  rhosvd_c2t_als_workspace_size(cp, opts, sweeps) bytes (the RHOSVD's plus the
 *              r_max^2-column contraction C_l and its Gram partials; 0 for invalid arguments,
 *              sweeps outside 0 .. RHOSVD_ALS_MAX_SWEEPS included)
 * Errors as rhosvd_c2t; RHOSVD_ERR_INVALID_ARG for sweeps outside 0 .. RHOSVD_ALS_MAX_SWEEPS.
 */
#define RHOSVD_ALS_MAX_SWEEPS 8
size_t rhosvd_c2t_als_workspace_size(const rhosvd_cp* cp, const rhosvd_opts* opts, int sweeps);
int rhosvd_c2t_als(const rhosvd_cp* cp, const rhosvd_opts* opts, int sweeps, const rhosvd_tucker* out,
                   double* energy, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Hadamard (entrywise) product of two canonical tensors with equal mode sizes
 * (Sec. 3 eq. rho_ten; Lemma 4.2): term nu = i + Ra * j of the result has columns
 * u^(l)_nu = a^(l)_i .* b^(l)_j and weight xa_i * xb_j; rank Ra * Rb.
 * U_out[l]: n_l x (Ra Rb), leading dimension ld_out[l] >= n_l; xi_out: Ra Rb values.
 * Output buffers must not overlap the inputs.
 */
int rhosvd_cp_hadamard(const rhosvd_cp* a, const rhosvd_cp* b, double* const U_out[3],
                       const int ld_out[3], double* xi_out, void* stream);

/*
 * Linear combination alpha A + beta B as one canonical tensor of rank Ra + Rb (Sec. 4.3:
 * sums are formed by grouping the terms): columns [A | B], weights [alpha xa | beta xb].
 */
int rhosvd_cp_sum(double alpha, const rhosvd_cp* a, double beta, const rhosvd_cp* b,
                  double* const U_out[3], const int ld_out[3], double* xi_out, void* stream);

/*
 * RHOSVD of the Hadamard product a (.) b without storing it (Sec. 3 eq. rho_ten reduced by
 * Def. 2.2): the same result as rhosvd_cp_hadamard into a buffer followed by rhosvd_c2t of that
 * buffer, bit for bit, but the norms and the normalised side matrices are formed from the columns
 * a^(l)_i .* b^(l)_j (term nu = i + Ra j, weight xa_i xb_j) as they are read, so the n_l x Ra Rb
 * product factors are never written to or read back from memory.  `out` is as for rhosvd_c2t
 * with R = Ra Rb (V: r_max x Ra Rb, xi_out: Ra Rb values).  Equal mode sizes; Ra Rb < 2^31.
 * Workspace: rhosvd_c2t_hadamard_workspace_size(a, b, opts) bytes (that of rhosvd_c2t for a
 * tensor of rank Ra Rb).  Errors as rhosvd_c2t.
 */
size_t rhosvd_c2t_hadamard_workspace_size(const rhosvd_cp* a, const rhosvd_cp* b, const rhosvd_opts* opts);
int rhosvd_c2t_hadamard(const rhosvd_cp* a, const rhosvd_cp* b, const rhosvd_opts* opts, const rhosvd_tucker* out,
                        void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------- allocation-free variant
 * (the paper has no counterpart: this serves callers of the library, not the method)
 *
 * rhosvd_c2t needs a device workspace from the caller.  Callers that cannot allocate device
 * memory -- code inside a host application that owns all device allocations, code that must
 * not risk the device-wide synchronisation cudaMalloc/cudaFree may bring, code with no
 * allocator at hand -- call rhosvd_c2t_noalloc instead: the same reduction, same arguments
 * minus the workspace, with scratch space taken from one static device array of
 * RHOSVD_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until exit.
 *   - Problems with rhosvd_c2t_workspace_size() > RHOSVD_NOALLOC_SCRATCH_BYTES are rejected
 *     with RHOSVD_ERR_SCRATCH_LIMIT; invalid arguments give RHOSVD_ERR_INVALID_ARG.
 *   - The first call on a device looks the array's address up (once per device); make that
 *     first call before any stream capture starts.  The address is kept per device ordinal,
 *     so the entry point assumes each device's primary runtime context: after cudaDeviceReset
 *     or under another context made current through the driver API it must not be called.
 *   - All calls on a device share the array and it keeps the previous call's contents (the
 *     reduction clears what it needs itself).  Calls that overlap on the GPU race on it:
 *     serialise them.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine.  (Tracing, if switched
 *     on with rhosvd_profile_enable, creates CUDA event objects on first use.)
 * Inputs and outputs are as for rhosvd_c2t; the caller still provides the output buffers. */
#define RHOSVD_NOALLOC_SCRATCH_BYTES (64u << 20)

int rhosvd_c2t_noalloc(const rhosvd_cp* cp, const rhosvd_opts* opts, const rhosvd_tucker* out,
                       void* stream);

/* ---------------------------------------------------------------- batched form (no paper
 * counterpart: many independent reductions, e.g. the Hartree-like products of many pairs)
 *
 * rhosvd_c2t_batched reduces `count` independent canonical tensors cps[i] with options
 * opts[i] into outs[i] (each as rhosvd_c2t would; results are identical to one rhosvd_c2t
 * call per tensor).  The tensors may have any n and R.  The library schedules them onto
 * `lanes` concurrent stream lanes (longest-processing-time first on the cost 3 (n1+n2+n3) R,
 * plus a fixed term for the sequential small factorisations); it captures the whole launch
 * sequence into one CUDA graph, caches the executable graph under the call's arguments (the
 * pointer values included), and launches it on `stream`.  A repeated call with the same
 * arguments is one graph launch.
 *   - lanes > 0: that many lanes (at most 32).  lanes <= 0: the library picks the count, by
 *     timing the candidates 4, 8, 16, 32 once on the first call for a batch shape (that first
 *     call synchronises the device), and remembers the fastest for that shape.
 *   - workspace: caller-owned device memory of rhosvd_c2t_batched_workspace_size(count, cps,
 *     opts, lanes) bytes, 256-byte aligned: one slot per lane, sized for the largest tensor.
 *   - Returns host-side argument errors like rhosvd_c2t; device-side conditions are in each
 *     outs[i].info.  Not reentrant across threads (one internal lock).
 *   - rhosvd_batch_latency_enable(1) makes later batched calls record, after each tensor, its
 *     completion time since the batch started; rhosvd_batch_latency_read(ms, count) waits for
 *     the last batch and writes those times (ms) in tensor order. */
size_t rhosvd_c2t_batched_workspace_size(int count, const rhosvd_cp* cps, const rhosvd_opts* opts, int lanes);
int rhosvd_c2t_batched(int count, const rhosvd_cp* cps, const rhosvd_opts* opts, const rhosvd_tucker* outs,
                       void* workspace, size_t workspace_bytes, int lanes, void* stream);
int rhosvd_batch_latency_enable(int on);
int rhosvd_batch_latency_read(float* ms, int count);

/* ---------------------------------------------------------------- learned subspace proposal
 * (no paper counterpart: a learned start for the range finder of the side-matrix SVD, eq.
 * SVD_Ul; the plain method stays its fallback and measures the error either way)
 *
 * rhosvd_c2t_start is rhosvd_c2t with the random range sketch replaced by a caller's start
 * basis Q0^(l) (n_l x k0, column-major, leading dimension ld[l] >= n_l, device): iters = 0 takes
 * Y = Q0 (no pass over U), iters = 1 one subspace iteration Y = U~ (U~^T Q0) (it scales each
 * direction by its sigma^2, so directions far below the largest fade from a Gram-based basis:
 * for a start that is already accurate use 0).  The rest is unchanged, the second (deflation)
 * sketch included, and so is the acceptance test: the measured energy outside the basis must
 * stay within eps^2 ||U~||^2 (energy captured >= 1 - eps^2), otherwise info.status is
 * RHOSVD_ERR_SKETCH and the caller falls back to rhosvd_c2t.  Modes with n_l <= r_max +
 * oversample keep the exact identity basis.  Workspace: rhosvd_c2t_start_workspace_size. */
size_t rhosvd_c2t_start_workspace_size(const rhosvd_cp* cp, const rhosvd_opts* opts, int k0);
int rhosvd_c2t_start(const rhosvd_cp* cp, const rhosvd_opts* opts, const double* const Q0[3], const int ld[3],
                     int k0, int iters, const rhosvd_tucker* out, void* workspace, size_t workspace_bytes,
                     void* stream);

/* The proposal network: 128 -> 512 -> 512 -> 512 -> 2048 with GELU (erf form) after the hidden
 * layers; FP32 master weights, BF16 copies for the GEMMs (tcgen05 tensor cores, FP32
 * accumulation); Adam (0.9, 0.999, 1e-8).  Input per mode: the 128 features of rhosvd_features.
 * Output per mode: 2048 = 64 x 32 values, C(i, j) at [i + 64 j], the coefficients of 32 vectors
 * over the Chebyshev polynomials T_0..T_63 of the grid (rhosvd_chebyshev); the proposal is
 * Q0 = T C.  Training loss per sample: ||C C^T - G||_F^2 averaged over the batch, with G (64 x 64
 * at [i + 64 i']) the target projector T^T Z Z^T T of the plain method's leading basis Z.
 * All device pointers are FP32 unless stated; batches are multiples of 8, at most batch_max.
 * The handle owns the weights (device memory); calls on one handle are serialised. */
int rhosvd_mlp_create(int batch_max, unsigned long long seed, void** handle);
int rhosvd_mlp_destroy(void* handle);
int rhosvd_mlp_forward(void* handle, const float* X, int B, float* Y, void* stream);
int rhosvd_mlp_gradients(void* handle, const float* X, const float* G, int B, float* loss, void* stream);
int rhosvd_mlp_train_step(void* handle, const float* X, const float* G, int B, float lr, float* loss, void* stream);
long long rhosvd_mlp_num_params(void);
/* host <-> device copy of all parameters (W0, b0, W1, b1, ...; W row-major out x in):
 * get = 1 reads (which = 0: the weights, 1: the gradients of the last rhosvd_mlp_gradients),
 * get = 0 writes the weights.  Synchronises the device. */
int rhosvd_mlp_params(void* handle, float* host, int get, int which);
/* Checkpoint / resume of the network's training state.  rhosvd_mlp_save writes, to the file
 * `path` (host path, created or truncated), a flat little-endian binary record: the 8-byte tag
 * "RHMLPv01", the layer count and the five layer widths (int32), the Adam step count (int64),
 * then per layer l the FP32 arrays W_l (out x in, row-major), b_l, the Adam moments m(W_l),
 * v(W_l), m(b_l), v(b_l).  rhosvd_mlp_load reads such a file into an existing handle (any
 * batch_max), restoring weights, moments and step, so that training resumes exactly where it
 * stopped; a file with another tag, other widths or a short body is rejected with
 * RHOSVD_ERR_INVALID_ARG and leaves the handle unchanged.  Both synchronise the device; file
 * errors return RHOSVD_ERR_INVALID_ARG. */
int rhosvd_mlp_save(void* handle, const char* path);
int rhosvd_mlp_load(void* handle, const char* path);
/* Status of the network's tensor-core products launched since the last call: synchronises
 * `stream`, returns RHOSVD_ERR_TIMEOUT if a bounded wait inside one of them expired (its
 * output is then not valid), else RHOSVD_OK; clears the record. */
int rhosvd_mlp_status(void* handle, void* stream);
/* Features of one Gaussian sum sum_k c_k exp(-a_k |x - x_k|^2) (device, FP64): per mode l,
 * out[128 l + 0..63] = c-weighted histogram (unit sum, 64 bins) of the centre coordinate x_{k,l}
 * over [-cbox, cbox], out[128 l + 64..127] = of log a_k over [la, lb] (values outside the range
 * fall into the end bins).  centres: R x 3 row-major; loga, c: length R; out: 3 x 128 FP32. */
int rhosvd_features(const double* centres, const double* loga, const double* c, int R, double cbox, double la,
                    double lb, float* out, void* stream);
/* Q_T (n x 64, column-major, device FP64, n >= 64): the Chebyshev polynomials T_j(x_i / b) on the
 * grid x_i = -b + (i + 1/2) 2b/n, orthonormalised in order (Gram-Schmidt twice per column): the
 * discrete orthogonal polynomials of the grid, the coordinates of the proposal. */
int rhosvd_chebyshev(int n, double b, double* T, void* stream);
/* Training target of one mode: G (64 x 64, FP32, G[i + 64 i']) = P P^T with P = Q_T^T Z, Z the
 * plain method's leading basis (n x r, column-major, ld ldz, r <= 64), all device memory. */
int rhosvd_proj_target(int n, const double* Q, const double* Z, int ldz, int r, float* G, void* stream);
/* The proposal of one mode: Q0 (n x 32, column-major, ld n, FP64) = Q_T C with C(i, j) = Y[i + 64 j]
 * the network's output for that mode (FP32). */
int rhosvd_proposal_basis(int n, const double* QT, const float* Y, double* Q0, void* stream);

/* ---------------------------------------------------------------- Tucker-to-canonical transform
 * (Sec. 2.4, Remark rem_can_red, eqs. T2C_slice, T2C_SVD, beta_R)
 *
 * rhosvd_t2c turns a Tucker tensor A = beta x_1 Z1 x_2 Z2 x_3 Z3 into a canonical one by the
 * SVDs of the core's slices along the third mode, B_m = beta(:, :, m):
 *   A_R = sum_m sum_{k <= p_m} sigma_k(B_m) (Z1 u_k) (x) (Z2 v_k) (x) Z3(:, m),
 * keeping the singular values above delta = eps ||beta||_F / (r3 sqrt(min(r1, r2))) (the
 * remark's eps / r^{3/2} for an r x r x r core, eps relative), so ||beta - beta_R||_F <=
 * eps ||beta||_F and, for orthonormal Z_l, ||A - A_R||_F is the same.  Canonical rank
 * R = sum_m p_m <= r3 min(r1, r2).  The C2C reduction is rhosvd_c2t followed by rhosvd_t2c.
 *
 *   t          the Tucker tensor (device pointers; Z_l column-major, n_l x r_l, ld ldz[l] >= n_l;
 *              beta r1 x r2 x r3 with entry (i, j, m) at beta[i + r1 (j + r2 m)], as rhosvd_c2t
 *              writes it); r1 r2 <= RHOSVD_T2C_SLICE_MAX and r1, r2 <= 1024 (a slice is
 *              factorised in one block's shared memory)
 *   eps        relative accuracy, >= 0 (0 keeps every singular value above the slice's FP64
 *              resolution min(r1, r2) u ||B_m||_F; values at or below it count as zero)
 *   R_max      capacity of the outputs (columns); U[l] n_l x R_max with leading dimension
 *              ldu[l] >= n_l, xi R_max (device, caller-owned)
 *   R_out      device int: the canonical rank R (also when it exceeds R_max)
 *   p_out      device int[r3] (may be NULL): p_m per slice
 *   status     device int: RHOSVD_OK, or RHOSVD_ERR_RANK_OVERFLOW when R > R_max (then U and xi
 *              are not written)
 *   workspace  device, >= rhosvd_t2c_workspace_size(t) bytes, 256-byte aligned
 * Host-side checks return RHOSVD_ERR_INVALID_ARG / RHOSVD_ERR_WORKSPACE; asynchronous on
 * `stream`.  Each slice's SVD: a Householder QR with column pivoting, then one-sided Jacobi on
 * the rows of R (bounded to 40 sweeps; about 8 on the bench's core), kept left vectors
 * re-orthonormalised. */
#define RHOSVD_T2C_SLICE_MAX 25600
typedef struct {
    int n[3];
    int r[3];
    const double* Z[3];
    int ldz[3];
    const double* beta;
} rhosvd_tucker_in;
size_t rhosvd_t2c_workspace_size(const rhosvd_tucker_in* t);
int rhosvd_t2c(const rhosvd_tucker_in* t, double eps, int R_max, double* const U[3], const int ldu[3], double* xi,
               int* R_out, int* p_out, int* status, void* workspace, size_t bytes, void* stream);

/* ---------------------------------------------------------------- polynomials of a canonical tensor
 * (Sec. 5: the tensor-valued polynomial P(A) = a_0 I + a_1 A + ... + a_n A^n of a reference
 * tensor, products taken entrywise, evaluated by the Horner scheme with the RHOSVD)
 *
 * rhosvd_cp_horner sets Y_n = a_n I (I the all-ones tensor, a rank-one term) and, for k = n-1
 * down to 0,
 *     Y_k = C2C( A (.) Y_{k+1} + a_k I ),
 * (.) the Hadamard product in rhosvd_cp_hadamard's term order (term i + R_A j), the constant
 * appended as the last term (left out when a_k = 0), and C2C = rhosvd_c2t with `opts` followed by
 * rhosvd_t2c with eps_t2c: one product and one reduction per degree.  Trailing zero coefficients
 * are dropped (the degree is that of the last nonzero a_k; the zero polynomial gives R = 0, a
 * constant gives the rank-one a_0 I without a reduction).  With exact reductions Y_0 = P(A);
 * otherwise Y_0 - P(A) = sum_k A^k (.) E_k, E_k the error of reduction k.
 *
 *   A          the reference tensor (device factors and weights, as for rhosvd_c2t)
 *   coeffs     host array a_0 .. a_{ncoeffs-1}, finite; ncoeffs >= 1
 *   opts       options of every RHOSVD; r_max^2 <= RHOSVD_T2C_SLICE_MAX
 *   eps_t2c    relative accuracy of every T2C, >= 0
 *   R_max      canonical capacity: every Y_k must have rank <= R_max (R_max >= 1)
 *   U_out, ldu, xi_out  device, caller-owned: U_out[l] n_l x R_max (ld ldu[l] >= n_l), xi_out R_max
 *              values; they hold each Y_k in turn and the result Y_0 at the end
 *   R_out      host int: the rank of Y_0 (columns 0 .. R_out-1 of U_out)
 *   steps      host array of ncoeffs - 1 records (may be NULL), one per reduction in the order
 *              k = n-1 .. 0: the rank R_in entering it, the Tucker ranks r, the canonical rank R
 *              and the step's status
 *   workspace  device, >= rhosvd_cp_horner_workspace_size(A, ncoeffs, opts, R_max) bytes, 256-byte
 *              aligned (it holds the product of rank R_A R_max + 1 and the RHOSVD and T2C scratch)
 * Returns RHOSVD_OK or the first error: INVALID_ARG, WORKSPACE or CUDA from the host checks, or
 * the device status of a reduction (RANK_OVERFLOW when a Tucker rank exceeds r_max or a canonical
 * rank exceeds R_max, NOT_CONVERGED, NONFINITE, SKETCH, TIMEOUT), with the records up to the
 * failing step filled.  The ranks of each step size the next launches, so the call synchronises
 * `stream` twice per degree and returns with the stream idle. */
typedef struct rhosvd_horner_step {
    int k;                  /* the coefficient index of this step                          */
    int R_in;               /* rank of A (.) Y_{k+1} + a_k I                               */
    int r[3];               /* Tucker ranks of its RHOSVD                                  */
    int R;                  /* canonical rank of Y_k after T2C                             */
    int status;             /* RHOSVD_OK or the step's device status                       */
} rhosvd_horner_step;
size_t rhosvd_cp_horner_workspace_size(const rhosvd_cp* A, int ncoeffs, const rhosvd_opts* opts, int R_max);
int rhosvd_cp_horner(const rhosvd_cp* A, const double* coeffs, int ncoeffs, const rhosvd_opts* opts,
                     double eps_t2c, int R_max, double* const U_out[3], const int ldu[3], double* xi_out,
                     int* R_out, rhosvd_horner_step* steps, void* workspace, size_t bytes, void* stream);

/* ---------------------------------------------------------------- entries at nodes and the
 * interaction energy from a long-range potential (Sec. 4.2, Lemma lem:InterEnergy, eq.
 * EnergyFree_Tensor)
 *
 * rhosvd_cp_sample writes the entries of the canonical tensor `cp` at N grid nodes:
 *   out[j] = sum_k xi_k U1[i1_j, k] U2[i2_j, k] U3[i3_j, k],  i_l,j = idx[l N + j]
 * (idx: device int array of 3 N zero-based grid indices, mode-major; out: device, N doubles).
 * A node whose index leaves [0, n_l) gets NaN (no memory outside the factors is read).
 *
 * rhosvd_rs_energy evaluates, for N charges z_j (device) sitting on the nodes idx of the grid of
 * the collective long-range potential P_long = sum_j z_j (shifted long-range reference kernel),
 *   E_N = 1/2 sum_j z_j P_long(x_j) - 1/2 p0 sum_j z_j^2,
 * where p0 = P_{R_l}(0) is the single reference kernel's long-range part at its own centre (host
 * double).  P_long may be the generated N R_l-term sum or its RHOSVD/C2C reduction; the work is
 * O(R N).  p_out (device, N doubles) receives the samples P_long(x_j); energy (device, 1 double)
 * the result.  Both calls are asynchronous on `stream`; sums run in a fixed order, so results do
 * not depend on the launch.  Errors: RHOSVD_ERR_INVALID_ARG (sizes, NULL pointers, non-finite
 * p0), RHOSVD_ERR_CUDA. */
int rhosvd_cp_sample(const rhosvd_cp* cp, int N, const int* idx, double* out, void* stream);
int rhosvd_rs_energy(const rhosvd_cp* P_long, int N, const int* idx, const double* z, double p0, double* p_out,
                     double* energy, void* stream);

/* ---------------------------------------------------------------- numerics self-test (no paper
 * counterpart: test support)
 *
 * rhosvd_selftest_fastmath evaluates, for n device doubles x, the short-latency reciprocal and
 * reciprocal square root the small factorisations use on their serial chains (an FP32
 * estimate of the exponent-scaled argument refined by two Newton-Raphson steps in FP64):
 * rcp[i] ~ 1/x[i], rsq[i] ~ 1/sqrt(x[i]) (device arrays of n doubles, caller-owned).  Returns
 * RHOSVD_ERR_INVALID_ARG for n < 0 or null pointers with n > 0; asynchronous on `stream`. */
int rhosvd_selftest_fastmath(const double* x, double* rcp, double* rsq, int n, void* stream);

/* rhosvd_selftest_bits evaluates, for n elements, the conversions the tensor-core products'
 * epilogues and the normalisation build from the bits instead of FP64 instructions:
 * rh[i] + rl[i] ~ x[i] (rh = x truncated to 24 significant bits, rl the rest rounded to a float:
 * within 2^-48 |x| for |x| >= 2^-97, 2^-120 below; both 0 for |x| < 2^-126), fd[i] = f[i] 2^e[i] exactly as a double (0 below FP64's normal
 * range), p2[i] = 2^e[i] as a float (subnormal from 2^-149, 0 below, infinity above 2^127).
 * Inputs x (doubles), f (floats), e (ints) and outputs rh, rl, p2 (floats), fd (doubles) are
 * device arrays of n elements, caller-owned.  Returns RHOSVD_ERR_INVALID_ARG for n < 0 or null
 * pointers with n > 0; asynchronous on `stream`. */
int rhosvd_selftest_bits(const double* x, const float* f, const int* e, float* rh, float* rl, double* fd,
                         float* p2, int n, void* stream);

/* FP64 rate probe (no paper counterpart: measurement support; the denominators of the FP64
 * rooflines are measured with it).  Launches `blocks` blocks of 256 threads, each thread
 * running eight independent FP64 fma chains of `iters` steps: 4096 * iters FLOP a block.
 * out: device array of blocks * 256 doubles (caller-owned) receiving each thread's chain sum.
 * Time it with events on `stream`.  RHOSVD_ERR_INVALID_ARG for blocks outside [1, 2^20],
 * iters < 1 or a null `out`. */
int rhosvd_probe_fp64(int blocks, int iters, double* out, void* stream);

/* ---------------------------------------------------------------- tracing (no paper
 * counterpart: observability of the library itself) */

/* Replayable call sequences (no paper counterpart: serving the same shapes repeatedly).
 * rhosvd_graph_begin starts capturing the library calls made on `stream` by this thread (a
 * created stream, not the legacy NULL stream) into a CUDA graph; rhosvd_graph_end stops, builds
 * the executable graph and returns its handle; rhosvd_graph_launch replays every captured kernel
 * on `stream` with the pointers of the capture (new inputs go into the same buffers);
 * rhosvd_graph_destroy frees it.  Calls whose ranks size later launches on the host
 * (rhosvd_cp_horner, rhosvd_c2t_als with energies) cannot be captured; every call that keeps its
 * ranks on the device (rhosvd_c2t, its fused, start and ALS forms without energies, the
 * products and sums, rhosvd_t2c, the energy) can.  Stage timing must be off or filtered while
 * capturing.  Errors: RHOSVD_ERR_INVALID_ARG (NULL stream or handle, nested capture),
 * RHOSVD_ERR_CUDA. */
int rhosvd_graph_begin(void* stream);
int rhosvd_graph_end(void* stream, void** graph);
int rhosvd_graph_launch(void* graph, void* stream);
int rhosvd_graph_destroy(void* graph);

/* Number of CUDA kernel launches the library has made since it was loaded (all threads). */
long long rhosvd_launch_count(void);

/* Turn per-stage timing on (1) or off (0); returns the previous setting.  When on, every
 * stage of rhosvd_c2t / rhosvd_cp_hadamard / rhosvd_cp_sum is bracketed by two CUDA events
 * recorded on the call's stream (the events come from a pool the library creates on first
 * use; at most 4096 stages are kept between reads). */
int rhosvd_profile_enable(int on);

/* Restrict the per-stage timing to the stages named `stage` (a copy of at most 63 characters is
 * kept; NULL or "" times every stage again).  With a filter, the other stages record no events,
 * so one kernel can be timed inside a timed region without perturbing the rest. */
int rhosvd_profile_filter(const char* stage);

/* Keep (1) the recorded stage events across rhosvd_profile_read instead of clearing them, so that
 * the events a graph capture recorded (see rhosvd_graph_begin: while capturing, a stage's events
 * become record nodes that every replay executes) can be read after each replay; 0 clears the
 * records.  Returns the previous setting. */
int rhosvd_profile_keep(int on);

/* Wait for the recorded events, then write one line "stage count total_ms" per stage into
 * buf (host memory, len bytes, NUL-terminated when it fits) and clear the records.
 * Returns the number of bytes written, or RHOSVD_ERR_CUDA. */
int rhosvd_profile_read(char* buf, int len);

#ifdef __cplusplus
}
#endif

#endif /* RHOSVD_H */

// internal.cuh -- shared definitions of the RHOSVD CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/rhosvd.h"

namespace rh {

constexpr int KMAX = RHOSVD_K_MAX;

// Per-call device state written and read by the kernels of one rhosvd_c2t call.
struct DevState {
    int kin[3];         // sketch width k_l (or n_l in the direct mode)
    int m[3];           // width of the orthonormal basis Q^(l) after rank revealing
    int r[3];           // Tucker ranks (mirror of info->r)
    int piv_fail[3];    // small factorisation break-down flags
    int rhi[3];         // number of leading eigenvectors computed (rank candidates 0..rhi)
    int r0[3];          // provisional rank from the eigenvalues
    int kx[3];          // columns of the current CholeskyQR input
    int kdef[3];        // width of the deflation sketch (second range sketch)
    int mdef[3];        // deflation directions kept
    int kxdef[3];       // columns of the deflation CholeskyQR input
    int near[3];        // the last Cholesky of the basis took the near-identity path (W written)
    int neardef[3];     // the same for the deflation basis
    double gmax[3];     // largest diagonal of the first sketch's Gram (scale of the sketch)
    double shift[3];    // shift used for the LDL^T representation of the tridiagonal
    double trace[3];    // trace(B B^T) = ||B||_F^2
    double total[3];    // ||U^(l) normalised||_F^2
    double rho2[3];     // ||U - Z_hi V_hi||_F^2, energy outside the rhi leading directions
    double specmax[3];  // upper bound of the spectrum of L D L^T
    int core_split;     // split-K count of the tensor-core Khatri-Rao core (from the ranks)
};

// Counter-based sign generator for the Rademacher sketch: bit (c & 63) of
// splitmix64(seed ^ (mode << 56) ^ (nu * 4 + (c >> 6))).  splitmix64 is Vigna's public
// 64-bit finaliser: add 0x9E3779B97F4A7C15, then two xor-shift-multiply rounds.
__host__ __device__ inline uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// the sign as a bit (1: +1), for producers that must stay off the FP64 pipe
__host__ __device__ inline int rademacher_bit(uint64_t seed, int mode, long long nu, int c)
{
    uint64_t h = splitmix64(seed ^ ((uint64_t)mode << 56) ^ ((uint64_t)nu * 4ull + (uint64_t)(c >> 6)));
    return (int)((h >> (c & 63)) & 1ull);
}

__host__ __device__ inline double rademacher(uint64_t seed, int mode, long long nu, int c)
{
    return rademacher_bit(seed, mode, nu, c) ? 1.0 : -1.0;
}

__device__ inline double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum; `red` must hold blockDim.x/32 doubles.  All threads get the result.  Warp 0
// adds the warp partials by a shuffle tree and broadcasts through shared memory: FP64 adds are
// slow on this part, and every thread adding all partials itself cost more than the data pass
// in a large block.
__device__ inline double block_sum(double v, double* red)
{
    __shared__ double bcast;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const double t = warp_sum(lane < nw ? red[lane] : 0.0);
        if (lane == 0) bcast = t;
    }
    __syncthreads();
    return bcast;
}

__device__ inline double block_max(double v, double* red)
{
    __shared__ double bcast;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const double t = warp_max(lane < nw ? red[lane] : 0.0);
        if (lane == 0) bcast = t;
    }
    __syncthreads();
    return bcast;
}

// Short-latency reciprocal and reciprocal square root for serial FP64 chains.  Dependent FP64
// operations are slow on this part, and the IEEE division and square root are long sequences;
// these take an FP32 estimate of the exponent-scaled argument (exact scaling by a power of two
// through the exponent field) and refine it by Newton-Raphson iterations in FP64:
//   1/d:        y <- y + y (1 - d y)                 (error squares each step)
//   1/sqrt(s):  y <- y + y (1/2 - (s y / 2) y)       (error squares each step)
// Two steps take the FP32 estimate (relative error < 2^-22) below 2^-88 before rounding, so the
// results are within a few units in the last place of the correctly rounded values (checked
// against CUDA's 1/x and 1/sqrt(x) by rhosvd_selftest_fastmath).  Arguments outside the normal
// range, zeros, infinities and NaNs take the IEEE operation.
__device__ __forceinline__ double fast_rcp(double d)
{
    const int hi = __double2hiint(d), lo = __double2loint(d);
    const int be = (hi >> 20) & 0x7FF;
    if (be < 2 || be > 2044) return 1.0 / d;
    const double m = __hiloint2double((hi & 0x800FFFFF) | (1023 << 20), lo);      // d 2^(1023 - be), |m| in [1, 2)
    double y = (double)(1.0f / (float)m);
    y = fma(y, fma(-m, y, 1.0), y);
    y = fma(y, fma(-m, y, 1.0), y);
    return y * __hiloint2double((2046 - be) << 20, 0);                              // times 2^(1023 - be)
}

__device__ __forceinline__ double fast_rsqrt(double s)
{
    const int hi = __double2hiint(s), lo = __double2loint(s);
    const int be = (hi >> 20) & 0x7FF;
    if (s <= 0.0 || be < 2 || be > 2044) return 1.0 / sqrt(s);
    const int e = be - 1023, h = e >> 1;                       // s = m 2^(2h), m in [1, 4)
    const double m = __hiloint2double((hi & 0x000FFFFF) | ((1023 + e - 2 * h) << 20), lo);
    double y = (double)rsqrtf((float)m);
    double hm = 0.5 * m;
    y = fma(y, fma(-hm * y, y, 0.5), y);
    y = fma(y, fma(-hm * y, y, 0.5), y);
    return y * __hiloint2double((1023 - h) << 20, 0);                                // times 2^-h
}

// Record the first device-side error in the info record.
__device__ inline void set_status(rhosvd_info* info, int code)
{
    atomicCAS(&info->status, 0, code);
}

// ---------------------------------------------------------------- generic FP64 GEMM
// C(i,j) (M x N) = sum_k A(i,k) B(k,j), one problem per "batch" (the three modes).
// Element (i,k) of a plain operand lives at p[i*rs + k*cs].
struct Mat {
    const double* p;
    long long rs, cs;
};

enum BKind { B_PLAIN = 0, B_SKETCH = 1, B_KR = 2 };

struct GemmProblem {
    Mat A, B;                  // B unused for generated kinds
    double* C;                 // output, element (i,j) at C[i*crs + j*ccs]
    long long crs, ccs;
    long long split_stride;    // offset between split-K partial outputs
    const double* colscale;    // nullable: C(:,j) *= colscale[j] in the epilogue
    const double* rowscale;    // nullable: C(i,:) *= rowscale[i]
    const int* dM;             // nullable device dims (ranks decided on the device)
    const int* dN;
    const int* dK;
    int M, N, K;               // host upper bounds (grid) / values when d* is NULL
    int N_from_r2r3;           // core: N = r2 * r3 taken from dNa, dNb
    const int* dNa;
    const int* dNb;
    // generated-B parameters
    const double* bscale;      // sketch: optional scale per row nu of B (null = 1)
    uint64_t seed;
    int mode;
    const double* V2;          // KR: B(nu, j + r2 m) = xi_nu V2(j,nu) V3(m,nu)
    const double* V3;
    const double* xi;
    int ldv;
    // residual-energy epilogue: instead of storing C, accumulate
    // sum (ref(i,j) * rscale[j] - C(i,j))^2 per thread block into rpart[tile]
    const double* rref;
    long long rref_ld;
    const double* rscale;      // null = 1
    double* rpart;
};

struct GemmBatch {
    GemmProblem p[3];
    int nbatch;
    int ksplit;
    int bkind;
};


// Maps blockIdx (0..nb-1) to the mode it works on, so a launch can cover any subset of modes.
struct ModeMap {
    int m[3];
};

// ---------------------------------------------------------------- kernel arguments
// v[l] of a three-entry kernel-parameter array at a runtime index l.  Indexing the array itself
// makes the compiler copy the whole parameter struct to local memory in every thread (a stack
// frame of a few hundred bytes a thread); a select chain reads the parameter bank directly.
template <typename T>
__device__ __forceinline__ T sel3(const T (&v)[3], int l)
{
    return l == 0 ? v[0] : (l == 1 ? v[1] : v[2]);
}

struct NormArgs {
    const double* U[3];
    int ld[3];
    int n[3];
    int R;
    double* norms;      // 3 x R
    double* colmax;     // 3 x R: max |u_i| of each column
    // Hadamard-product source (Ra > 0): column nu = i + Ra j is U[l](:, i) .* B[l](:, j) and its
    // weight xa[i] xb[j], formed on the fly (the same FP64 products rhosvd_cp_hadamard stores)
    const double* B[3];
    int ldb[3];
    int Ra;
    const double* xa;
    const double* xb;
};

// Digit planes of the normalised columns, cut while they are written (mixed form): column nu
// of mode l becomes operand row nu (k = x) with its own exponent.  planes[l] null: none.
struct NormSlice {
    uint16_t* planes[3];
    long long pstride[3];
    int ld[3];
    signed char* exps[3];
    int tiles_k[3];            // > 0: tile-major planes with this many k tiles (see ozgemm.cuh)
    int tile_h[3];             // their rows per tile
};

struct HadArgs {
    const double* A[3];
    int lda[3];
    const double* B[3];
    int ldb[3];
    double* C[3];
    int ldc[3];
    int n[3];
    int Ra, Rb;
    const double* xa;
    const double* xb;
    double* xc;
};

struct SumArgs {
    const double* A[3];
    int lda[3];
    const double* B[3];
    int ldb[3];
    double* C[3];
    int ldc[3];
    int n[3];
    int Ra, Rb;
    const double* xa;
    const double* xb;
    double* xc;
    double alpha, beta;
};


struct RankArgs {
    const double* mu;
    int vstride;
    const int* dk;
    const double* trace;     // per mode
    const double* total;     // per mode
    double eps;
    int ranks[3];
    int r_max;
    double* sigma[3];        // user outputs (KMAX each)
    rhosvd_info* info;
    DevState* st;
    int direct[3];
    const int* kept;         // info->kept
    int margin;              // extra candidate directions beyond the provisional rank
};

struct FinalArgs {
    const double* V;         // rhi x R per mode, ld ldv
    long long vstride;
    int ldv;
    int R;
    double eps;
    int ranks[3];
    int r_max;
    rhosvd_info* info;
    DevState* st;
    const double* rpart;     // residual partials per mode
    int ntiles[3];
    long long rpstride;
    double* cpart;           // Ritz energy partials: [mode][chunk][KMAX]
    int nchunk;              // chunks of nu (at most RITZ_CHUNKS)
    int n[3];                // mode sizes (the FP64 noise floor of a mode's energies)
};
constexpr int RITZ_CHUNKS = 256;

// Transposed digit planes with a fixed exponent (the range-sketch operand: rows x, k = nu).
struct SliceTArgs {
    const double* X[3];
    int ldx[3];
    int rows[3];
    int K[3];
    uint16_t* planes[3];
    long long pstride[3];
    int ld[3];
    int E0;
    int tiles_k[3];            // > 0: tile-major planes with this many k tiles (see ozgemm.cuh)
    int tile_h[3];             // their rows per tile
    int S;                     // digits: 0 or 7 (the FP64-class seven), or 5 (OZ_SKETCH5)
};

// The range sketch's Rademacher signs as a tile-major BF16 plane (rows j = sketch column, k = nu).
struct SignPlaneArgs {
    uint16_t* planes[3];
    int rows[3];               // sketch width k_l
    int K[3];                  // R
    int mode[3];
    int tiles_k;               // k tiles (16 wide) of every plane
    unsigned long long seed;
};
int launch_sign_planes(const SignPlaneArgs& a, int nb, int rowsmax, cudaStream_t st);

struct DeflDims {
    int n[3];
    const int* dm;     // device basis widths
};

// ---------------------------------------------------------------- launchers (return 0 or RHOSVD_ERR_CUDA)
int launch_gemm(GemmBatch& gb, cudaStream_t st);
int launch_gemm_splitk(GemmBatch gb, double* part, cudaStream_t st);
int launch_colnorms(const NormArgs& a, cudaStream_t st);
int launch_terms(const NormArgs& na, const double* xi, double* keepf, double* xin, double* xi_user,
                 rhosvd_info* info, double* Un, long long ustride, double* nn2, double* total, const NormSlice& ns,
                 cudaStream_t st);
int launch_identity(double* Q, int n, int ld, cudaStream_t st);
int launch_slice_t(const SliceTArgs& a, int nb, int ldmax, int rowsmax, cudaStream_t st);
int launch_row_exps(const float2* Vp, long long vstride, int ldp, const int* dr, int mode0, int nmodes, int R,
                    signed char* out, long long ostride, cudaStream_t st);
int launch_split_v(const double* src, long long sstride, int lds, float2* dst, long long dstride, int ldd, int R,
                   const int* dr, int mode0, int nmodes, cudaStream_t st);
int launch_init_state(DevState* s, int k0, int k1, int k2, int m0, int m1, int m2, int kdef, cudaStream_t st);
int launch_hadamard(const HadArgs& a, cudaStream_t st);
int launch_cpsum(const SumArgs& a, cudaStream_t st);
// With a near-identity Gram the factor's inverse is written to W directly (the layout of
// launch_trinv) and near_out[b] = 1, which launch_trinv then skips; else near_out[b] = 0.
int launch_chol(ModeMap mm, const double* G, long long gstride, int ldg, const int* dk, int* kx_out, double* L,
                long long lstride, int ldl, int* perm, int pstride, int* dm_out, int* fail, int pivot, double tol, int nb,
                int kbound, double* d0_out, const double* d0_ref, double floor_rel, double* W, long long wstride,
                int ldw, int* near_out, cudaStream_t st);
// Deflation of the second range sketch against the basis Q (n x m, ld n per mode):
// T = Q^T Y, then Y -= Q T (k2 columns of Y, ld n).
int launch_deflate(ModeMap mm, const double* Q, double* Y, long long nk, const int n[3], const int* dm, int k2,
                   double* T, long long tstride, int nb, int nmax, cudaStream_t st);
// Q(:, m + j) = Q2(:, j), j < m2 (device counts), then m += m2.
int launch_append(ModeMap mm, double* Q, const double* Q2, long long nk, const int n[3], int* dm, const int* dm2,
                  int nb, int nmax, int k2, cudaStream_t st);
int launch_trinv(ModeMap mm, const double* L, long long lstride, int ldl, const int* perm, int pstride,
                 const int* dkx, const int* dm, double* W, long long wstride, int ldw, const int* near, int nb,
                 cudaStream_t st);
int launch_trace(ModeMap mm, const double* A, long long astride, int lda, const int* dk, double* trace, int nb,
                 cudaStream_t st);
int launch_tridiag(ModeMap mm, double* A, long long astride, int lda, const int* dk, double* d, double* e, double* tau,
                   int vstride, int nb, int kbound, cudaStream_t st);
// The pivoted Cholesky and the tridiagonal reduction on a thread-block cluster per mode
// (cluster.cu); kbound <= KMAX.
int launch_chol_cluster(ModeMap mm, const double* G, long long gstride, int ldg, const int* dk, int* kx_out, double* L,
                        long long lstride, int ldl, int* perm, int pstride, int* dm_out, int* fail, int pivot,
                        double tol, int nb, int kbound, double* d0_out, const double* d0_ref, double floor_rel,
                        double* W, long long wstride, int ldw, int* near_out, cudaStream_t st);
int launch_tridiag_cluster(ModeMap mm, double* A, long long astride, int lda, const int* dk, double* d, double* e,
                           double* tau, int vstride, int nb, int kbound, cudaStream_t st);
int launch_eigvals(ModeMap mm, const double* d, const double* e, int vstride, const int* dk, double* D, double* Lo,
                   double* mu, DevState* s, int nb, cudaStream_t st);
int launch_rank(const RankArgs& a, cudaStream_t st);
int launch_rank_final(const FinalArgs& a, cudaStream_t st);
int launch_copy2d(const double* src, long long sstride, const int lds[3], double* const dst[3], const int ldd[3],
                  const int* drows, const int hrows[3], const int* dcols, const int hcols[3], cudaStream_t st);
// FP32 outputs: dst[b][e] = (float)src[b][e] (round to nearest) for e < cnt[b], or, where cnt[b]
// < 0, for e < dr[0] dr[1] dr[2] (the packed core of device ranks dr).  nb <= 4.
int launch_to_f32(const double* const src[4], float* const dst[4], const long long cnt[4], const int* dr, int nb,
                  cudaStream_t st);
int launch_eigvecs(ModeMap mm, const double* D, const double* Lo, const double* mu, int vstride, const int* dk,
                   const DevState* s, double* W, long long wstride, int ldw, int rmax, int nb, cudaStream_t st);
int launch_backtransform(ModeMap mm, const double* A, long long astride, int lda, const double* tau, int vstride,
                         const int* dk, const DevState* s, double* W, long long wstride, int ldw, int rmax,
                         int nb, cudaStream_t st);

// ALS refinement helpers (als.cu): step sizes and the captured energy before/after a mode step
int launch_als_set(DevState* s, int l, int* kk, cudaStream_t st);
int launch_als_energy_before(const double* G, int ldg, const double* W, int ldw, const int* dm, const int* dr,
                             int rmax, double* part, double* out, cudaStream_t st);
int launch_als_energy_after(const double* mu, const DevState* s, int l, double* out, cudaStream_t st);

}  // namespace rh

namespace rh {
void count_launch();   // library-wide kernel launch counter (rhosvd_launch_count)
}

#define RH_CHECK_LAUNCH()                                   \
    do {                                                    \
        rh::count_launch();                                 \
        cudaError_t e_ = cudaGetLastError();                \
        if (e_ != cudaSuccess) return RHOSVD_ERR_CUDA;      \
    } while (0)

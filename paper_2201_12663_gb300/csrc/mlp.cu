// mlp.cu -- the learned subspace proposal: a small MLP maps a per-mode summary of a Gaussian
// sum (c-weighted histograms of the centre coordinate and of the log-exponent) to NCOEF
// coefficient vectors over NCHEB Chebyshev polynomials of the grid; their span seeds the range
// finder (rhosvd_c2t_start), with the plain method as the fallback when the captured energy is
// short of 1 - eps^2.
//
// Network: 128 -> 512 -> 512 -> 512 -> 2048, GELU (erf form) after the hidden layers, FP32 master
// weights with BF16 copies for the GEMMs, which run on the tcgen05 tensor cores (the digit-plane
// kernel with one plane per operand, FP32 accumulation).  Activations and gradients are FP32.
// Loss per sample: || C C^T - G ||_F^2 with C (64 x 32) the reshaped output and G = T^T Z Z^T T
// the target projector of the plain RHOSVD's leading basis in Chebyshev coordinates (invariant
// to the signs and rotations of Z).  Adam on the FP32 master weights.
#include "internal.cuh"
#include "ozgemm.cuh"

#include <cuda_bf16.h>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

namespace rh {
namespace {

constexpr int NL = 4;                                   // layers
constexpr int DIMS[NL + 1] = {128, 512, 512, 512, 2048};
constexpr int NCHEB = 64, NCOEF = 32, NBIN = 64;

__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&b);
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// standard normal from a counter hash (Box-Muller on two 53-bit uniforms)
__device__ __forceinline__ double hash_normal(unsigned long long seed, unsigned long long i)
{
    const uint64_t a = splitmix64(seed ^ (2 * i)), b = splitmix64(seed ^ (2 * i + 1));
    const double u1 = ((a >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (b >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// W (out x in, row-major) ~ N(0, 2 / in), bias 0
__global__ void k_init(float* W, float* b, int out, int in, unsigned long long seed)
{
    const long long total = (long long)out * in;
    const double sd = sqrt(2.0 / in);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        W[e] = (float)(sd * hash_normal(seed, (unsigned long long)e));
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < out; e += gridDim.x * blockDim.x) b[e] = 0.f;
}

// dst (bf16, rows x cols, ld) = src (fp32, rows x cols, lds), or its transpose (trans: dst is
// cols x rows with ld, dst(j, i) = src(i, j))
__global__ void k_to_bf16(const float* src, int rows, int cols, int lds, uint16_t* dst, int ld, int trans)
{
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / cols), j = (int)(e % cols);
        const uint16_t v = bf16_bits(src[(long long)i * lds + j]);
        if (trans) dst[(long long)j * ld + i] = v;
        else dst[(long long)i * ld + j] = v;
    }
}

// pre = C + bias (fp32), act = gelu(pre) (or pre for the last layer)
__global__ void k_bias_act(const double* C, const float* bias, int rows, int cols, float* pre, float* act, int last)
{
    const long long total = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const float z = (float)C[e] + bias[e % cols];
        pre[e] = z;
        act[e] = last ? z : gelu(z);
    }
}

// dZ = dA * gelu'(pre)
__global__ void k_gelu_back(const float* dA, const float* pre, float* dZ, long long total)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        dZ[e] = dA[e] * gelu_grad(pre[e]);
}

// db(j) = sum_b dZ(b, j); grad(fp32) = (float) Cdouble for dW.  One thread per column.
__global__ void k_colsum(const float* dZ, int rows, int cols, float* db)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int b = 0; b < rows; ++b) s += dZ[(long long)b * cols + j];
    db[j] = s;
}

__global__ void k_d2f(const double* src, float* dst, long long total)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        dst[e] = (float)src[e];
}

// loss and its gradient, one block per sample: C(i, j) = Y[b, i + 64 j], D = C C^T - G_b,
// loss_b = ||D||^2, dY[b, i + 64 j] = (4 / B) sum_i' D(i, i') C(i', j)
__global__ void k_proj_loss(const float* Y, const float* G, int B, float* dY, float* loss_b)
{
    const int b = blockIdx.x;
    __shared__ float C[NCHEB * NCOEF];
    __shared__ float D[NCHEB * NCHEB];
    __shared__ float red[32];
    const float* y = Y + (long long)b * NCHEB * NCOEF;
    for (int e = threadIdx.x; e < NCHEB * NCOEF; e += blockDim.x) C[e] = y[e];
    __syncthreads();
    const float* g = G + (long long)b * NCHEB * NCHEB;
    float l2 = 0.f;
    for (int e = threadIdx.x; e < NCHEB * NCHEB; e += blockDim.x) {
        const int i = e % NCHEB, i2 = e / NCHEB;
        float s = 0.f;
        for (int j = 0; j < NCOEF; ++j) s += C[i + NCHEB * j] * C[i2 + NCHEB * j];
        const float d = s - g[e];
        D[e] = d;
        l2 += d * d;
    }
    __syncthreads();
    const float sc = 4.0f / B;
    for (int e = threadIdx.x; e < NCHEB * NCOEF; e += blockDim.x) {
        const int i = e % NCHEB, j = e / NCHEB;
        float s = 0.f;
        for (int i2 = 0; i2 < NCHEB; ++i2) s += D[i + NCHEB * i2] * C[i2 + NCHEB * j];
        dY[(long long)b * NCHEB * NCOEF + e] = sc * s;
    }
    // block sum of l2
    for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        loss_b[b] = t;
    }
}

__global__ void k_mean(const float* x, int n, float* out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += x[i];
    *out = (float)(s / n);
}

// Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, w -= lr mhat / (sqrt(vhat) + 1e-8)
__global__ void k_adam(float* w, const float* g, float* m, float* v, long long total, float lr, float c1, float c2)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = 0.9f * m[e] + 0.1f * gi;
        const float vi = 0.999f * v[e] + 0.001f * gi * gi;
        m[e] = mi;
        v[e] = vi;
        w[e] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
    }
}

// Features of one tensor's mode l: c-weighted histograms (unit sum) of the centre coordinate
// over [-cbox, cbox] and of log a over [la, lb], 64 bins each, out[l * 128 + 0..63] and
// [64..127].  One thread per bin loops over the terms (deterministic).  grid (3), block 128.
__global__ void k_features(const double* centres, const double* loga, const double* c, int R, double cbox,
                           double la, double lb, float* out)
{
    const int l = blockIdx.x, t = threadIdx.x;
    const bool is_c = t < NBIN;
    const int bin = is_c ? t : t - NBIN;
    const double lo = is_c ? -cbox : la, hi = is_c ? cbox : lb;
    double s = 0.0, tot = 0.0;
    for (int k = 0; k < R; ++k) {
        const double x = is_c ? centres[(long long)k * 3 + l] : loga[k];
        int q = (int)floor((x - lo) / (hi - lo) * NBIN);
        q = q < 0 ? 0 : (q >= NBIN ? NBIN - 1 : q);
        tot += c[k];
        if (q == bin) s += c[k];
    }
    out[l * 2 * NBIN + t] = tot > 0.0 ? (float)(s / tot) : 0.f;
}

// T (n x 64, column-major, ld n): T_j(x_i / b) on the cell-centre grid x_i = -b + (i + 1/2) 2b/n
__global__ void k_chebyshev(int n, double b, double* T)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = (-b + (i + 0.5) * 2.0 * b / n) / b;
    double t0 = 1.0, t1 = x;
    T[i] = t0;
    if (NCHEB > 1) T[(long long)n + i] = t1;
    for (int j = 2; j < NCHEB; ++j) {
        const double t2 = 2.0 * x * t1 - t0;
        T[(long long)j * n + i] = t2;
        t0 = t1;
        t1 = t2;
    }
}

// Orthonormalise the 64 columns in order (classical Gram-Schmidt applied twice per column, then
// normalisation): the discrete orthogonal polynomials of the grid.  One block of 256 threads.
__global__ void k_cheb_orth(int n, double* Q)
{
    __shared__ double d[NCHEB];
    __shared__ double red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = 0; j < NCHEB; ++j) {
        double* qj = Q + (long long)j * n;
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            for (int i = warp; i < j; i += 8) {
                const double* qi = Q + (long long)i * n;
                double s = 0.0;
                for (int x = lane; x < n; x += 32) s = fma(qi[x], qj[x], s);
                s = warp_sum(s);
                if (lane == 0) d[i] = s;
            }
            __syncthreads();
            for (int x = threadIdx.x; x < n; x += blockDim.x) {
                double v = qj[x];
                for (int i = 0; i < j; ++i) v = fma(-d[i], Q[(long long)i * n + x], v);
                qj[x] = v;
            }
            __syncthreads();
        }
        double s = 0.0;
        for (int x = threadIdx.x; x < n; x += blockDim.x) s = fma(qj[x], qj[x], s);
        s = warp_sum(s);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        double nrm2 = 0.0;
        for (int w = 0; w < 8; ++w) nrm2 += red[w];
        const double inv = 1.0 / sqrt(nrm2);
        __syncthreads();
        for (int x = threadIdx.x; x < n; x += blockDim.x) qj[x] *= inv;
        __syncthreads();
    }
}

// G (64 x 64, FP32, G[i + 64 i']) = P P^T with P = Q^T Z (64 x r): one block; P in shared memory
__global__ void k_proj_target(int n, const double* Q, const double* Z, int ldz, int r, float* G)
{
    __shared__ double P[NCHEB * 64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int e = warp; e < NCHEB * r; e += nw) {
        const int i = e % NCHEB, j = e / NCHEB;
        const double* qi = Q + (long long)i * n;
        const double* zj = Z + (long long)j * ldz;
        double s = 0.0;
        for (int x = lane; x < n; x += 32) s = fma(qi[x], zj[x], s);
        s = warp_sum(s);
        if (lane == 0) P[i + NCHEB * j] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NCHEB * NCHEB; e += blockDim.x) {
        const int i = e % NCHEB, i2 = e / NCHEB;
        double s = 0.0;
        for (int j = 0; j < r; ++j) s = fma(P[i + NCHEB * j], P[i2 + NCHEB * j], s);
        G[e] = (float)s;
    }
}

// Q0 (n x 32, column-major, ld n) = Q_T (n x 64) C, C(i, j) = Y[i + 64 j] (FP32).  Thread per entry.
__global__ void k_proposal(int n, const double* QT, const float* Y, double* Q0)
{
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * NCOEF) return;
    const int x = (int)(e % n), j = (int)(e / n);
    double s = 0.0;
    for (int i = 0; i < NCHEB; ++i) s = fma(QT[(long long)i * n + x], (double)Y[i + NCHEB * j], s);
    Q0[e] = s;
}

int grid_for(long long total) { return (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096); }

struct Mlp {
    int bmax = 0;
    int step = 0;
    float *W[NL] = {}, *b[NL] = {}, *mW[NL] = {}, *vW[NL] = {}, *mb[NL] = {}, *vb[NL] = {};
    float *gW[NL] = {}, *gb[NL] = {};
    uint16_t *Wbf[NL] = {}, *WTbf[NL] = {};
    // per-layer activations for the batch: input A_i (fp32 and bf16, plus transposed bf16)
    float* act[NL + 1] = {};
    float* pre[NL] = {};
    uint16_t *Abf[NL] = {}, *ATbf[NL] = {};
    float *dA = nullptr, *dZ = nullptr;
    uint16_t *dZbf = nullptr, *dZTbf = nullptr;
    double* Cd = nullptr;
    float* lossb = nullptr;
    void* pool = nullptr;
};

std::mutex g_mlp_mu;

// C (M x N, row-major, double) = A (M x K bf16, ld K) B (N x K bf16, ld K)^T on the tensor cores
int bf16_gemm(const uint16_t* A, int M, const uint16_t* B, int N, int K, double* C, cudaStream_t st)
{
    OzBatch ob;
    memset(&ob, 0, sizeof(ob));
    ob.nbatch = 1;
    ob.err = nullptr;
    OzProblem& q = ob.p[0];
    q.A = OzPlanes{A, 0, K, nullptr, 8};
    q.B = OzPlanes{B, 0, K, nullptr, 8};
    q.M = M;
    q.N = N;
    q.K = K;
    q.C = C;
    q.crs = N;
    q.ccs = 1;
    return launch_ozgemm(ob, OZ_BF16, st);
}

int forward(Mlp* m, const float* X, int B, cudaStream_t st)
{
    if (cudaMemcpyAsync(m->act[0], X, sizeof(float) * (size_t)B * DIMS[0], cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    for (int i = 0; i < NL; ++i) {
        const int in = DIMS[i], out = DIMS[i + 1];
        k_to_bf16<<<grid_for((long long)B * in), 256, 0, st>>>(m->act[i], B, in, in, m->Abf[i], in, 0);
        RH_CHECK_LAUNCH();
        k_to_bf16<<<grid_for((long long)B * in), 256, 0, st>>>(m->act[i], B, in, in, m->ATbf[i], B, 1);
        RH_CHECK_LAUNCH();
        int rc = bf16_gemm(m->Abf[i], B, m->Wbf[i], out, in, m->Cd, st);
        if (rc) return rc;
        k_bias_act<<<grid_for((long long)B * out), 256, 0, st>>>(m->Cd, m->b[i], B, out, m->pre[i], m->act[i + 1],
                                                                  i == NL - 1);
        RH_CHECK_LAUNCH();
    }
    return 0;
}

int refresh_bf16(Mlp* m, cudaStream_t st)
{
    for (int i = 0; i < NL; ++i) {
        const int in = DIMS[i], out = DIMS[i + 1];
        k_to_bf16<<<grid_for((long long)out * in), 256, 0, st>>>(m->W[i], out, in, in, m->Wbf[i], in, 0);
        RH_CHECK_LAUNCH();
        k_to_bf16<<<grid_for((long long)out * in), 256, 0, st>>>(m->W[i], out, in, in, m->WTbf[i], out, 1);
        RH_CHECK_LAUNCH();
    }
    return 0;
}

void destroy(Mlp* m)
{
    if (m->pool) cudaFree(m->pool);
    delete m;
}

}  // namespace
}  // namespace rh

using namespace rh;

extern "C" int rhosvd_mlp_create(int batch_max, unsigned long long seed, void** handle)
{
    if (!handle || batch_max < 8 || batch_max % 8 != 0) return RHOSVD_ERR_INVALID_ARG;
    Mlp* m = new Mlp();
    m->bmax = batch_max;
    size_t off = 0;
    std::vector<std::pair<void**, size_t>> req;
    auto want = [&](void** p, size_t bytes) { req.push_back({p, bytes}); };
    for (int i = 0; i < NL; ++i) {
        const size_t wsz = (size_t)DIMS[i] * DIMS[i + 1];
        for (float** p : {&m->W[i], &m->mW[i], &m->vW[i], &m->gW[i]}) want((void**)p, sizeof(float) * wsz);
        for (float** p : {&m->b[i], &m->mb[i], &m->vb[i], &m->gb[i]}) want((void**)p, sizeof(float) * DIMS[i + 1]);
        want((void**)&m->Wbf[i], 2 * wsz);
        want((void**)&m->WTbf[i], 2 * wsz);
        want((void**)&m->pre[i], sizeof(float) * (size_t)batch_max * DIMS[i + 1]);
        want((void**)&m->Abf[i], 2 * (size_t)batch_max * DIMS[i]);
        want((void**)&m->ATbf[i], 2 * (size_t)batch_max * DIMS[i]);
    }
    for (int i = 0; i <= NL; ++i) want((void**)&m->act[i], sizeof(float) * (size_t)batch_max * DIMS[i]);
    want((void**)&m->dA, sizeof(float) * (size_t)batch_max * 2048);
    want((void**)&m->dZ, sizeof(float) * (size_t)batch_max * 2048);
    want((void**)&m->dZbf, 2 * (size_t)batch_max * 2048);
    want((void**)&m->dZTbf, 2 * (size_t)batch_max * 2048);
    want((void**)&m->Cd, sizeof(double) * (size_t)batch_max * 2048 > sizeof(double) * 2048 * 512
                             ? sizeof(double) * (size_t)batch_max * 2048 : sizeof(double) * 2048 * 512);
    want((void**)&m->lossb, sizeof(float) * (size_t)batch_max);
    for (auto& r : req) off += (r.second + 255) / 256 * 256;
    if (cudaMalloc(&m->pool, off) != cudaSuccess) { delete m; return RHOSVD_ERR_CUDA; }
    cudaMemset(m->pool, 0, off);
    char* base = (char*)m->pool;
    size_t o = 0;
    for (auto& r : req) { *r.first = base + o; o += (r.second + 255) / 256 * 256; }
    for (int i = 0; i < NL; ++i) {
        k_init<<<256, 256>>>(m->W[i], m->b[i], DIMS[i + 1], DIMS[i], seed + 7919ull * i);
        count_launch();
    }
    if (refresh_bf16(m, 0) || cudaDeviceSynchronize() != cudaSuccess) { destroy(m); return RHOSVD_ERR_CUDA; }
    *handle = m;
    return 0;
}

extern "C" int rhosvd_mlp_destroy(void* handle)
{
    if (!handle) return RHOSVD_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    destroy((Mlp*)handle);
    return 0;
}

extern "C" int rhosvd_mlp_forward(void* handle, const float* X, int B, float* Y, void* stream)
{
    Mlp* m = (Mlp*)handle;
    if (!m || !X || !Y || B < 1 || B > m->bmax || B % 8 != 0) return RHOSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    int rc = forward(m, X, B, st);
    if (rc) return rc;
    if (cudaMemcpyAsync(Y, m->act[NL], sizeof(float) * (size_t)B * DIMS[NL], cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    return 0;
}

extern "C" int rhosvd_mlp_gradients(void* handle, const float* X, const float* G, int B, float* loss, void* stream)
{
    Mlp* m = (Mlp*)handle;
    if (!m || !X || !G || !loss || B < 8 || B > m->bmax || B % 8 != 0) return RHOSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    int rc = forward(m, X, B, st);
    if (rc) return rc;
    k_proj_loss<<<B, 256, 0, st>>>(m->act[NL], G, B, m->dA, m->lossb);
    RH_CHECK_LAUNCH();
    k_mean<<<1, 32, 0, st>>>(m->lossb, B, loss);
    RH_CHECK_LAUNCH();
    for (int i = NL - 1; i >= 0; --i) {
        const int in = DIMS[i], out = DIMS[i + 1];
        const long long tot = (long long)B * out;
        if (i == NL - 1) {
            if (cudaMemcpyAsync(m->dZ, m->dA, sizeof(float) * tot, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                return RHOSVD_ERR_CUDA;
        } else {
            k_gelu_back<<<grid_for(tot), 256, 0, st>>>(m->dA, m->pre[i], m->dZ, tot);
            RH_CHECK_LAUNCH();
        }
        k_colsum<<<(out + 255) / 256, 256, 0, st>>>(m->dZ, B, out, m->gb[i]);
        RH_CHECK_LAUNCH();
        k_to_bf16<<<grid_for(tot), 256, 0, st>>>(m->dZ, B, out, out, m->dZbf, out, 0);
        RH_CHECK_LAUNCH();
        k_to_bf16<<<grid_for(tot), 256, 0, st>>>(m->dZ, B, out, out, m->dZTbf, B, 1);
        RH_CHECK_LAUNCH();
        // dW (out x in) = dZ^T A: rows o of dZ^T (k = batch) against rows j of A^T (k = batch)
        rc = bf16_gemm(m->dZTbf, out, m->ATbf[i], in, B, m->Cd, st);
        if (rc) return rc;
        k_d2f<<<grid_for((long long)out * in), 256, 0, st>>>(m->Cd, m->gW[i], (long long)out * in);
        RH_CHECK_LAUNCH();
        if (i > 0) {
            // dA (B x in) = dZ W: rows b of dZ (k = out) against rows j of W^T (k = out)
            rc = bf16_gemm(m->dZbf, B, m->WTbf[i], in, out, m->Cd, st);
            if (rc) return rc;
            k_d2f<<<grid_for((long long)B * in), 256, 0, st>>>(m->Cd, m->dA, (long long)B * in);
            RH_CHECK_LAUNCH();
        }
    }
    return 0;
}

extern "C" int rhosvd_mlp_train_step(void* handle, const float* X, const float* G, int B, float lr, float* loss,
                                     void* stream)
{
    int rc = rhosvd_mlp_gradients(handle, X, G, B, loss, stream);
    if (rc) return rc;
    Mlp* m = (Mlp*)handle;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    m->step += 1;
    const float c1 = 1.0f / (1.0f - powf(0.9f, (float)m->step)), c2 = 1.0f / (1.0f - powf(0.999f, (float)m->step));
    for (int i = 0; i < NL; ++i) {
        const long long wsz = (long long)DIMS[i] * DIMS[i + 1];
        k_adam<<<grid_for(wsz), 256, 0, st>>>(m->W[i], m->gW[i], m->mW[i], m->vW[i], wsz, lr, c1, c2);
        RH_CHECK_LAUNCH();
        k_adam<<<grid_for(DIMS[i + 1]), 256, 0, st>>>(m->b[i], m->gb[i], m->mb[i], m->vb[i], DIMS[i + 1], lr, c1, c2);
        RH_CHECK_LAUNCH();
    }
    return refresh_bf16(m, st);
}

// parameters in the order W0, b0, W1, b1, ...: host copies (get = 1) or uploads (get = 0);
// gradients (which = 1) of the last rhosvd_mlp_gradients call can be read the same way
extern "C" long long rhosvd_mlp_num_params(void)
{
    long long s = 0;
    for (int i = 0; i < NL; ++i) s += (long long)DIMS[i] * DIMS[i + 1] + DIMS[i + 1];
    return s;
}

extern "C" int rhosvd_mlp_params(void* handle, float* host, int get, int which)
{
    Mlp* m = (Mlp*)handle;
    if (!m || !host || (which != 0 && which != 1) || (which == 1 && !get)) return RHOSVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return RHOSVD_ERR_CUDA;
    size_t o = 0;
    for (int i = 0; i < NL; ++i) {
        const size_t wsz = (size_t)DIMS[i] * DIMS[i + 1];
        float* w = which ? m->gW[i] : m->W[i];
        float* b = which ? m->gb[i] : m->b[i];
        const cudaMemcpyKind k = get ? cudaMemcpyDeviceToHost : cudaMemcpyHostToDevice;
        if (cudaMemcpy(get ? (void*)(host + o) : (void*)w, get ? (void*)w : (void*)(host + o), sizeof(float) * wsz, k) !=
            cudaSuccess)
            return RHOSVD_ERR_CUDA;
        o += wsz;
        if (cudaMemcpy(get ? (void*)(host + o) : (void*)b, get ? (void*)b : (void*)(host + o),
                       sizeof(float) * DIMS[i + 1], k) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        o += DIMS[i + 1];
    }
    if (!get) {
        if (refresh_bf16(m, 0) || cudaDeviceSynchronize() != cudaSuccess) return RHOSVD_ERR_CUDA;
    }
    return 0;
}

namespace {
const char MLP_TAG[8] = {'R', 'H', 'M', 'L', 'P', 'v', '0', '1'};

// lengths of the six FP32 state arrays of layer i in file order: W, b, m(W), v(W), m(b), v(b)
void layer_lengths(int i, size_t len[6])
{
    const size_t wsz = (size_t)DIMS[i] * DIMS[i + 1], bsz = (size_t)DIMS[i + 1];
    const size_t l[6] = {wsz, bsz, wsz, wsz, bsz, bsz};
    for (int k = 0; k < 6; ++k) len[k] = l[k];
}

// the handle's device arrays of layer i in the same order
void layer_arrays(Mlp* m, int i, float* arr[6])
{
    float* a[6] = {m->W[i], m->b[i], m->mW[i], m->vW[i], m->mb[i], m->vb[i]};
    for (int k = 0; k < 6; ++k) arr[k] = a[k];
}
}  // namespace

extern "C" int rhosvd_mlp_save(void* handle, const char* path)
{
    Mlp* m = (Mlp*)handle;
    if (!m || !path) return RHOSVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return RHOSVD_ERR_CUDA;
    std::vector<float> host;
    FILE* f = fopen(path, "wb");
    if (!f) return RHOSVD_ERR_INVALID_ARG;
    int32_t hdr[NL + 2];
    hdr[0] = NL;
    for (int i = 0; i <= NL; ++i) hdr[1 + i] = DIMS[i];
    const int64_t step = m->step;
    bool ok = fwrite(MLP_TAG, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), NL + 2, f) == (size_t)(NL + 2) &&
              fwrite(&step, sizeof(step), 1, f) == 1;
    int rc = RHOSVD_OK;
    for (int i = 0; ok && i < NL; ++i) {
        float* arr[6];
        size_t len[6];
        layer_lengths(i, len);
        layer_arrays(m, i, arr);
        for (int k = 0; ok && k < 6; ++k) {
            host.resize(len[k]);
            if (cudaMemcpy(host.data(), arr[k], sizeof(float) * len[k], cudaMemcpyDeviceToHost) != cudaSuccess) {
                rc = RHOSVD_ERR_CUDA;
                ok = false;
                break;
            }
            ok = fwrite(host.data(), sizeof(float), len[k], f) == len[k];
        }
    }
    ok = (fclose(f) == 0) && ok;
    if (rc) return rc;
    return ok ? RHOSVD_OK : RHOSVD_ERR_INVALID_ARG;
}

extern "C" int rhosvd_mlp_load(void* handle, const char* path)
{
    Mlp* m = (Mlp*)handle;
    if (!m || !path) return RHOSVD_ERR_INVALID_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return RHOSVD_ERR_INVALID_ARG;
    // read and check the whole file before touching the handle
    char tag[8];
    int32_t hdr[NL + 2];
    int64_t step = 0;
    bool ok = fread(tag, 1, 8, f) == 8 && memcmp(tag, MLP_TAG, 8) == 0 &&
              fread(hdr, sizeof(int32_t), NL + 2, f) == (size_t)(NL + 2) && hdr[0] == NL &&
              fread(&step, sizeof(step), 1, f) == 1 && step >= 0 && step < (1LL << 40);
    for (int i = 0; ok && i <= NL; ++i) ok = hdr[1 + i] == DIMS[i];
    std::vector<std::vector<float>> body;
    for (int i = 0; ok && i < NL; ++i) {
        size_t len[6];
        layer_lengths(i, len);
        for (int k = 0; ok && k < 6; ++k) {
            body.emplace_back(len[k]);
            ok = fread(body.back().data(), sizeof(float), len[k], f) == len[k];
        }
    }
    if (ok) {                                 // nothing may follow the record
        char extra;
        ok = fread(&extra, 1, 1, f) == 0;
    }
    fclose(f);
    if (!ok) return RHOSVD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mlp_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return RHOSVD_ERR_CUDA;
    size_t q = 0;
    for (int i = 0; i < NL; ++i) {
        float* arr[6];
        size_t len[6];
        layer_lengths(i, len);
        layer_arrays(m, i, arr);
        for (int k = 0; k < 6; ++k, ++q)
            if (cudaMemcpy(arr[k], body[q].data(), sizeof(float) * len[k], cudaMemcpyHostToDevice) != cudaSuccess)
                return RHOSVD_ERR_CUDA;
    }
    m->step = (int)step;
    if (refresh_bf16(m, 0) || cudaDeviceSynchronize() != cudaSuccess) return RHOSVD_ERR_CUDA;
    return RHOSVD_OK;
}

extern "C" int rhosvd_mlp_status(void* handle, void* stream)
{
    if (!handle) return RHOSVD_ERR_INVALID_ARG;
    int v = 0;
    const int rc = oz_take_status((cudaStream_t)stream, &v);
    if (rc) return rc;
    return v ? RHOSVD_ERR_TIMEOUT : RHOSVD_OK;
}

extern "C" int rhosvd_features(const double* centres, const double* loga, const double* c, int R, double cbox,
                               double la, double lb, float* out, void* stream)
{
    if (!centres || !loga || !c || !out || R < 1 || !(cbox > 0.0) || !(lb > la)) return RHOSVD_ERR_INVALID_ARG;
    k_features<<<3, 2 * NBIN, 0, (cudaStream_t)stream>>>(centres, loga, c, R, cbox, la, lb, out);
    RH_CHECK_LAUNCH();
    return 0;
}

extern "C" int rhosvd_chebyshev(int n, double b, double* T, void* stream)
{
    if (n < NCHEB || !(b > 0.0) || !T) return RHOSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    k_chebyshev<<<(n + 127) / 128, 128, 0, st>>>(n, b, T);
    RH_CHECK_LAUNCH();
    k_cheb_orth<<<1, 256, 0, st>>>(n, T);
    RH_CHECK_LAUNCH();
    return 0;
}

extern "C" int rhosvd_proj_target(int n, const double* Q, const double* Z, int ldz, int r, float* G, void* stream)
{
    if (n < 1 || !Q || !Z || ldz < n || r < 1 || r > 64 || !G) return RHOSVD_ERR_INVALID_ARG;
    k_proj_target<<<1, 256, 0, (cudaStream_t)stream>>>(n, Q, Z, ldz, r, G);
    RH_CHECK_LAUNCH();
    return 0;
}

extern "C" int rhosvd_proposal_basis(int n, const double* QT, const float* Y, double* Q0, void* stream)
{
    if (n < 1 || !QT || !Y || !Q0) return RHOSVD_ERR_INVALID_ARG;
    const long long tot = (long long)n * NCOEF;
    k_proposal<<<(unsigned)((tot + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n, QT, Y, Q0);
    RH_CHECK_LAUNCH();
    return 0;
}

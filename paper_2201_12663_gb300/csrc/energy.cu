// energy.cu -- entries of a canonical tensor at grid nodes and the interaction energy of N
// charges from the long-range part of their collective potential (Sec. 4.2, Lemma
// lem:InterEnergy, eq. EnergyFree_Tensor):
//   p_l(j) = sum_k xi_k U1[i1_j, k] U2[i2_j, k] U3[i3_j, k],
//   E_N = 1/2 <z, p_l> - 1/2 P_{R_l}(0) sum_j z_j^2,
// O(R N) work for a rank-R (typically RHOSVD-reduced) potential.  Fixed reduction orders: the
// results do not depend on the launch.
#include "internal.cuh"
#include <math.h>

namespace rh {
namespace {

struct SampleArgs {
    const double* U[3];
    int ld[3];
    int n[3];
    int R;
    const double* xi;
    const int* idx;      // 3 x N, mode l at idx[l N + j]
    int N;
    double* out;
};

// one warp per node j: lane k-strided products ((xi_k u1) u2) u3, then the warp's fixed tree
__global__ void k_cp_sample(SampleArgs a)
{
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= a.N) return;
    const int i0 = a.idx[j], i1 = a.idx[a.N + j], i2 = a.idx[2 * a.N + j];
    const bool ok = i0 >= 0 && i0 < a.n[0] && i1 >= 0 && i1 < a.n[1] && i2 >= 0 && i2 < a.n[2];
    double s = 0.0;
    if (ok) {
        const double* u0 = a.U[0] + i0;
        const double* u1 = a.U[1] + i1;
        const double* u2 = a.U[2] + i2;
        for (int k = lane; k < a.R; k += 32)
            s += ((a.xi[k] * u0[(long long)k * a.ld[0]]) * u1[(long long)k * a.ld[1]]) * u2[(long long)k * a.ld[2]];
    }
    s = warp_sum(s);
    if (lane == 0) a.out[j] = ok ? s : __longlong_as_double(0x7FF8000000000000ll);
}

// one block: E = 1/2 sum z_j p_j - 1/2 p0 sum z_j^2
__global__ void k_rs_energy(const double* z, const double* p, int N, double p0, double* E)
{
    __shared__ double red[32];
    double s1 = 0.0, s2 = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        s1 = fma(z[j], p[j], s1);
        s2 = fma(z[j], z[j], s2);
    }
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) E[0] = 0.5 * s1 - 0.5 * p0 * s2;
}

int sample_args(const rhosvd_cp* cp, int N, const int* idx, double* out, SampleArgs* a)
{
    if (!cp || N < 0 || cp->R < 0) return RHOSVD_ERR_INVALID_ARG;
    if (N > 0 && (!idx || !out)) return RHOSVD_ERR_INVALID_ARG;
    for (int l = 0; l < 3; ++l) {
        if (cp->n[l] < 1 || cp->ld[l] < cp->n[l]) return RHOSVD_ERR_INVALID_ARG;
        if (cp->R > 0 && !cp->U[l]) return RHOSVD_ERR_INVALID_ARG;
        a->U[l] = cp->U[l];
        a->ld[l] = cp->ld[l];
        a->n[l] = cp->n[l];
    }
    if (cp->R > 0 && !cp->xi) return RHOSVD_ERR_INVALID_ARG;
    a->R = cp->R;
    a->xi = cp->xi;
    a->idx = idx;
    a->N = N;
    a->out = out;
    return RHOSVD_OK;
}

}  // namespace
}  // namespace rh

extern "C" int rhosvd_cp_sample(const rhosvd_cp* cp, int N, const int* idx, double* out, void* stream)
{
    rh::SampleArgs a;
    int rc = rh::sample_args(cp, N, idx, out, &a);
    if (rc) return rc;
    if (N == 0) return RHOSVD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    rh::k_cp_sample<<<(N + 7) / 8, 256, 0, st>>>(a);
    rh::count_launch();
    return cudaGetLastError() == cudaSuccess ? RHOSVD_OK : RHOSVD_ERR_CUDA;
}

extern "C" int rhosvd_rs_energy(const rhosvd_cp* P_long, int N, const int* idx, const double* z, double p0,
                                double* p_out, double* energy, void* stream)
{
    rh::SampleArgs a;
    int rc = rh::sample_args(P_long, N, idx, p_out, &a);
    if (rc) return rc;
    if (!energy || (N > 0 && !z) || !isfinite(p0)) return RHOSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (N > 0) {
        rh::k_cp_sample<<<(N + 7) / 8, 256, 0, st>>>(a);
        rh::count_launch();
    }
    rh::k_rs_energy<<<1, 1024, 0, st>>>(z, p_out, N, p0, energy);
    rh::count_launch();
    return cudaGetLastError() == cudaSuccess ? RHOSVD_OK : RHOSVD_ERR_CUDA;
}

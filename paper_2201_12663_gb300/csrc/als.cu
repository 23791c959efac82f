// als.cu -- small kernels of the canonical-to-Tucker ALS refinement that follows the RHOSVD
// (Sec. 2.2, eq. can_A_Tuck_als).  A mode-l step works inside the RHOSVD's orthonormal basis
// Q_l of the side matrix: with B_l = Q_l^T U~_l, the contraction of the canonical tensor with
// the other two factors has the unfolding Q_l C_l, C_l = B_l diag(xi') (V_m2 (.) V_m1)^T, and
// its best rank-r_l subspace is Q_l W_l with W_l the leading eigenvectors of G_l = C_l C_l^T.
// The GEMMs and the eigen-decomposition reuse the RHOSVD's kernels; these kernels set the
// step's sizes and record the captured energy ||beta||^2 before and after the step.
#include "internal.cuh"

namespace rh {
namespace {

// rhi[l] = r[l] (the ALS keeps the RHOSVD's ranks), kk[l] = r[m1] r[m2]
__global__ void k_als_set(DevState* s, int l, int m1, int m2, int* kk)
{
    s->rhi[l] = s->r[l];
    kk[l] = s->r[m1] * s->r[m2];
}

// part[j] = w_j^T G w_j for j < r (one block per j; G symmetric m x m, ld ldg; W ld ldw)
__global__ void k_als_quad(const double* G, int ldg, const double* W, int ldw, const int* dm, const int* dr,
                           double* part)
{
    __shared__ double red[32];
    const int j = blockIdx.x, m = *dm;
    if (j >= *dr) return;
    const double* w = W + (long long)j * ldw;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double t = 0.0;
        for (int c = 0; c < m; ++c) t = fma(G[(long long)c * ldg + i], w[c], t);
        s = fma(w[i], t, s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[j] = s;
}

// out = sum_{j < r} part[j] in index order
__global__ void k_als_sum(const double* part, const int* dr, double* out)
{
    double s = 0.0;
    for (int j = 0; j < *dr; ++j) s += part[j];
    *out = s;
}

// out = sum of the r largest eigenvalues max(mu[m-1-j] - shift, 0) of mode l
__global__ void k_als_top(const double* mu, const DevState* s, int l, double* out)
{
    const int m = s->m[l], r = s->r[l];
    double e = 0.0;
    for (int j = 0; j < r && j < m; ++j) e += fmax(mu[m - 1 - j] - s->shift[l], 0.0);
    *out = e;
}

}  // namespace

int launch_als_set(DevState* s, int l, int* kk, cudaStream_t st)
{
    const int m1 = l == 0 ? 1 : 0, m2 = l == 2 ? 1 : 2;
    k_als_set<<<1, 1, 0, st>>>(s, l, m1, m2, kk);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_als_energy_before(const double* G, int ldg, const double* W, int ldw, const int* dm, const int* dr,
                             int rmax, double* part, double* out, cudaStream_t st)
{
    if (rmax > 0) {
        k_als_quad<<<rmax, 256, 0, st>>>(G, ldg, W, ldw, dm, dr, part);
        RH_CHECK_LAUNCH();
    }
    k_als_sum<<<1, 1, 0, st>>>(part, dr, out);
    RH_CHECK_LAUNCH();
    return 0;
}

int launch_als_energy_after(const double* mu, const DevState* s, int l, double* out, cudaStream_t st)
{
    k_als_top<<<1, 1, 0, st>>>(mu, s, l, out);
    RH_CHECK_LAUNCH();
    return 0;
}

}  // namespace rh

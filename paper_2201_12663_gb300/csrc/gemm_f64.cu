// gemm_f64.cu -- batched FP64 GEMM on the CUDA cores for the plain (FP64) RHOSVD path.
//
// One launch covers the three modes (grid.z = batch x split-K).  The B operand is either a
// plain strided matrix, the Rademacher sketch matrix diag(1/||u_nu||) Omega generated from a
// counter-based hash (range sketch U Omega of the side matrix), or the Khatri-Rao operand
// xi_nu V2(j,nu) V3(m,nu) formed on the fly (core contraction of Prop. 2.2).
#include "internal.cuh"

namespace rh {

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

__device__ inline int dim_or(const int* d, int h) { return d ? *d : h; }

template <int KIND>
__global__ void __launch_bounds__(GT) k_gemm_f64(GemmBatch gb)
{
    const int b = blockIdx.z / gb.ksplit;
    const int s = blockIdx.z % gb.ksplit;
    const GemmProblem& P = gb.p[b];
    const int M = dim_or(P.dM, P.M);
    int N = dim_or(P.dN, P.N);
    if (P.N_from_r2r3) N = (*P.dNa) * (*P.dNb);
    const int K = dim_or(P.dK, P.K);
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    if (i0 >= M || j0 >= N) {
        if (P.rpart && threadIdx.x == 0) P.rpart[blockIdx.x + gridDim.x * blockIdx.y] = 0.0;
        return;
    }
    int kc = (K + gb.ksplit - 1) / gb.ksplit;
    kc = (kc + BK - 1) / BK * BK;
    const int kbeg = s * kc, kend = min(K, kbeg + kc);

    __shared__ double As[BK][BM];
    __shared__ double Bs[BK][BN + 1];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;

    const bool a_colmajor = (P.A.rs == 1);
    const bool b_kcontig = (KIND == B_PLAIN) ? (P.B.rs == 1) : false;
    int r2 = 1;
    if (KIND == B_KR) r2 = *P.dNa;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // ---- A tile (BM x BK)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int ii, kk;
            if (a_colmajor) { ii = t & 63; kk = (t >> 6) + 4 * q; }
            else { ii = (t >> 4) + 16 * q; kk = t & 15; }
            const int gi = i0 + ii, gk = k0 + kk;
            double v = 0.0;
            if (gi < M && gk < kend) v = P.A.p[(long long)gi * P.A.rs + (long long)gk * P.A.cs];
            As[kk][ii] = v;
        }
        // ---- B tile (BK x BN)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int kk, jj;
            if (KIND == B_PLAIN && b_kcontig) { kk = t & 15; jj = (t >> 4) + 16 * q; }
            else { jj = t & 63; kk = (t >> 6) + 4 * q; }
            const int gk = k0 + kk, gj = j0 + jj;
            double v = 0.0;
            if (gk < kend && gj < N) {
                if (KIND == B_PLAIN) {
                    v = P.B.p[(long long)gk * P.B.rs + (long long)gj * P.B.cs];
                } else if (KIND == B_SKETCH) {
                    const double sc = P.bscale ? P.bscale[gk] : 1.0;
                    v = (sc == 0.0) ? 0.0 : sc * rademacher(P.seed, P.mode, gk, gj);
                } else {
                    const int jm = gj / r2, jj2 = gj - jm * r2;
                    const long long off = (long long)gk * P.ldv;
                    v = P.xi[gk] * P.V2[off + jj2] * P.V3[off + jm];
                }
            }
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double a[4], bb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[kk][ty + 16 * q]; bb[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], bb[y], acc[x][y]);
        }
        __syncthreads();
    }
    if (P.rpart) {
        // residual energy of this tile: sum (ref(i,j) rscale[j] - C(i,j))^2
        double e2 = 0.0;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int gi = i0 + ty + 16 * x;
            if (gi >= M) continue;
#pragma unroll
            for (int y = 0; y < 4; ++y) {
                const int gj = j0 + tx + 16 * y;
                if (gj >= N) continue;
                const double v = P.rref[(long long)gi + P.rref_ld * gj] * (P.rscale ? P.rscale[gj] : 1.0) - acc[x][y];
                e2 = fma(v, v, e2);
            }
        }
        double* red = &As[0][0];
        e2 = block_sum(e2, red);
        if (t == 0) P.rpart[blockIdx.x + gridDim.x * blockIdx.y] = e2;
        return;
    }
    long long ccs = P.ccs;
    if (P.ccs < 0) ccs = M;  // core: column stride = r1 decided on the device
    double* C = P.C + (long long)s * P.split_stride;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int gi = i0 + ty + 16 * x;
        if (gi >= M) continue;
        const double rsc = P.rowscale ? P.rowscale[gi] : 1.0;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int gj = j0 + tx + 16 * y;
            if (gj >= N) continue;
            const double csc = P.colscale ? P.colscale[gj] : 1.0;
            C[(long long)gi * P.crs + (long long)gj * ccs] = acc[x][y] * rsc * csc;
        }
    }
}

// Sum split-K partials (contiguous M x N column-major blocks, stride `ss`) into C.
__global__ void k_reduce_splits(const double* part, long long ss, int ksplit, int Mmax, int Nmax,
                                const int* dM0, const int* dN0, double* C0, long long crs0, long long ccs0,
                                long long bstride_part, const int* dM1, const int* dN1, double* C1,
                                long long crs1, long long ccs1, const int* dM2, const int* dN2,
                                double* C2, long long crs2, long long ccs2, int Mh, int Nh)
{
    const int b = blockIdx.y;
    const int* dM = b == 0 ? dM0 : (b == 1 ? dM1 : dM2);
    const int* dN = b == 0 ? dN0 : (b == 1 ? dN1 : dN2);
    double* C = b == 0 ? C0 : (b == 1 ? C1 : C2);
    const long long crs = b == 0 ? crs0 : (b == 1 ? crs1 : crs2);
    const long long ccs = b == 0 ? ccs0 : (b == 1 ? ccs1 : ccs2);
    const int M = dM ? *dM : Mh, N = dN ? *dN : Nh;
    const double* P = part + (long long)b * bstride_part;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)M * N;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % M), j = (int)(e / M);
        double v = 0.0;
        for (int s = 0; s < ksplit; ++s) v += P[s * ss + (long long)i + (long long)j * Mmax];
        C[i * crs + j * ccs] = v;
    }
    (void)Nmax;
}

int launch_gemm(GemmBatch& gb, cudaStream_t st)
{
    int Mh = 0, Nh = 0;
    for (int b = 0; b < gb.nbatch; ++b) {
        Mh = max(Mh, gb.p[b].M);
        Nh = max(Nh, gb.p[b].N);
    }
    if (Mh <= 0 || Nh <= 0) return 0;
    dim3 grid((Mh + BM - 1) / BM, (Nh + BN - 1) / BN, gb.nbatch * gb.ksplit);
    if (grid.y > 65535) return RHOSVD_ERR_INVALID_ARG;
    switch (gb.bkind) {
    case B_PLAIN: k_gemm_f64<B_PLAIN><<<grid, GT, 0, st>>>(gb); break;
    case B_SKETCH: k_gemm_f64<B_SKETCH><<<grid, GT, 0, st>>>(gb); break;
    default: k_gemm_f64<B_KR><<<grid, GT, 0, st>>>(gb); break;
    }
    RH_CHECK_LAUNCH();
    return 0;
}

// Split-K GEMM whose partials go to `part` (capacity nbatch * ksplit * Mh * Nh doubles)
// and are then summed into each problem's C with its own strides.
int launch_gemm_splitk(GemmBatch gb, double* part, cudaStream_t st)
{
    int Mh = 0, Nh = 0;
    for (int b = 0; b < gb.nbatch; ++b) {
        Mh = max(Mh, gb.p[b].M);
        Nh = max(Nh, gb.p[b].N);
    }
    if (Mh <= 0 || Nh <= 0) return 0;
    GemmBatch g2 = gb;
    const long long ss = (long long)Mh * Nh;
    const long long bstride = ss * gb.ksplit;
    for (int b = 0; b < gb.nbatch; ++b) {
        g2.p[b].C = part + b * bstride;
        g2.p[b].crs = 1;
        g2.p[b].ccs = Mh;
        g2.p[b].split_stride = ss;
    }
    int rc = launch_gemm(g2, st);
    if (rc) return rc;
    const GemmProblem* p = gb.p;
    const int nb = gb.nbatch;
    dim3 grid(64, nb);
    k_reduce_splits<<<grid, 256, 0, st>>>(part, ss, gb.ksplit, Mh, Nh, p[0].dM, p[0].dN, p[0].C, p[0].crs,
                                          p[0].ccs, bstride, nb > 1 ? p[1].dM : nullptr,
                                          nb > 1 ? p[1].dN : nullptr, nb > 1 ? p[1].C : nullptr,
                                          nb > 1 ? p[1].crs : 0, nb > 1 ? p[1].ccs : 0,
                                          nb > 2 ? p[2].dM : nullptr, nb > 2 ? p[2].dN : nullptr,
                                          nb > 2 ? p[2].C : nullptr, nb > 2 ? p[2].crs : 0,
                                          nb > 2 ? p[2].ccs : 0, Mh, Nh);
    RH_CHECK_LAUNCH();
    return 0;
}

}  // namespace rh

// cluster.cu -- the small dense factorisations of one mode spread over a thread-block cluster.
//
// On this part the FP64 pipe issues about two fused multiply-adds per clock per SM, so a k x k
// factorisation held by one block (one SM per mode) is bound by that SM's FP64 issue.  Here C
// blocks of a cluster (16 where the device schedules such clusters, else the portable 8) share
// one mode: each owns the rows i = rank + li C of the trailing matrix, in full length, in its
// shared memory; the vectors every block needs are all-gathered through distributed shared
// memory, and a step's phases are separated by cluster barriers (hardware barriers, no
// spin-waits).  Every block computes the step's scalars itself from the same gathered values
// in the same order, so all blocks take identical branches and arrive at every barrier.
#include "internal.cuh"
#include <cooperative_groups.h>
#include <limits.h>

namespace cg = cooperative_groups;

namespace rh {

constexpr int TC_THREADS = 256;

// ------------------------------------------------------------------ tridiagonalisation
// Householder reduction of the symmetric k x k matrix A (full storage, ld lda, lower triangle
// read) to tridiagonal form.  Reflector j (j = 0..k-3): x = A(j+1:k, j),
// alpha = -sign(x_0) ||x||, v = x - alpha e_1, tau = 2 / v^T v; the trailing block gets
// A <- H A H via p = tau A v, w = p - (tau/2)(p^T v) v, A <- A - v w^T - w v^T.  Output: d
// (diagonal), e (sub-diagonal), tau, and v stored in A(j+1:k, j) for the back-transformation.
// Block `rank` holds rows i = rank + li C (full rows, ld k).  Every block also holds the step's
// pivot row x = A(j, j:k) (= column j by symmetry), the same in every block.  Per step, one
// cluster barrier:
//   B  every block forms alpha, tau and v from x (the same sums in the same order everywhere);
//      p_i = tau A(i, :) v for its rows and its part of p^T v, both kept locally; the owner of
//      row j+1 keeps a copy of that row as it stands before the update; cluster barrier;
//   C  every block reads p and the p^T v parts from their owners and the copy of row j+1, forms
//      w, updates its rows and applies the same update to the copy, which gives step j+1's pivot
//      row without a second exchange.
// Nothing is written into another block's memory: on GB300 a cluster barrier alone costs ~540
// cycles, ~1400 more with remote stores pending at it, and a round of remote loads after it
// ~1100; the step's loads go out together, in the one round its pivot row copy needs anyway.
// The update applies to element (i, c) and to its mirror (c, i) the same operations on the
// same operands, fma(-v_lo, w_hi, fma(-w_lo, v_hi, a)) with lo = min(i, c), hi = max(i, c), so
// the full-row storage stays exactly symmetric, and the pivot row every block rebuilds is the
// owner's row bit for bit.  The buffers read across blocks (p, the p^T v part, the row copy)
// alternate by step parity: a block writes step j+2's only after the barrier of step j+1, which
// no block passes before it has read step j's.
template <int C>
__global__ void __launch_bounds__(TC_THREADS) k_tridiag_cluster(ModeMap mm, double* A, long long astride, int lda,
                                                                const int* dk, double* d, double* e, double* tau,
                                                                int vstride)
{
    constexpr int ROWS = (KMAX + C - 1) / C;                       // rows a block owns at most
    constexpr int RP2 = ROWS <= 8 ? 8 : (ROWS <= 16 ? 16 : 32);    // ... rounded up to a power of two
    constexpr int NCH = TC_THREADS / RP2;                          // column chunks per row in A v
    static_assert(ROWS <= 32 && NCH >= 1 && NCH <= 32 && (NCH & (NCH - 1)) == 0, "row split");
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int b = mm.m[blockIdx.y];
    const int k = dk[b];
    A += b * astride;
    d += b * vstride;
    e += b * vstride;
    tau += b * vstride;
    extern __shared__ double Srow[];
    __shared__ double xg[KMAX], xn[KMAX], pg[KMAX], vl[KMAX], wl[KMAX], qloc[32];
    __shared__ double pown[2][32], nrow[2][KMAX], pvl[2];
    __shared__ double dsh[KMAX], esh[KMAX], tsh[KMAX];
    __shared__ double sc[4];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nloc = rank < k ? (k - rank + C - 1) / C : 0;
    // the owned rows from the lower triangle: A(i, c) = A[c lda + i] for c <= i, A[i lda + c] above
    for (int idx = tid; idx < nloc * k; idx += TC_THREADS) {
        const int li = idx / k, c = idx - li * k;
        const int i = rank + li * C;
        Srow[idx] = c <= i ? A[(long long)c * lda + i] : A[(long long)i * lda + c];
    }
    // the first pivot row, A(0, c) = A[c]
    for (int c = tid; c < k; c += TC_THREADS) xg[c] = A[c];
    cl.sync();                     // every block resident and loaded before the first remote access
    for (int j = 0; j + 2 < k; ++j) {
        const int c0 = j + 1, par = j & 1;
        const int li0 = c0 <= rank ? 0 : (c0 - rank + C - 1) / C;  // first owned row >= c0
        const int nr = nloc > li0 ? nloc - li0 : 0;
        // ---- B: the Householder scalars in the last warp while warps 0..6 form
        // q_i = sum_{c > c0} A(i, c) x_c for the owned rows: v differs from x only in entry c0,
        // so A v = q + A(:, c0) v0 needs no scalar until the end, and the scalar chain (a square
        // root and a reciprocal, long dependent FP64 sequences) runs beside the product
        if (warp == TC_THREADS / 32 - 1) {
            double s = 0.0;
            for (int c = c0 + 1 + lane; c < k; c += 32) s = fma(xg[c], xg[c], s);
            const double t2 = warp_sum(s);                        // same order in every block
            if (lane == 0) {
                const double x0 = xg[c0];
                double tj = 0.0, al = x0, v0 = 0.0;
                if (t2 != 0.0) {
                    const double s2 = fma(x0, x0, t2);
                    const double xn0 = s2 * fast_rsqrt(s2);
                    al = (x0 >= 0.0) ? -xn0 : xn0;
                    v0 = x0 - al;
                    tj = 2.0 * fast_rcp(fma(v0, v0, t2));
                }
                sc[0] = tj;
                sc[1] = al;
                sc[2] = v0;
                tsh[j] = tj;                           // outputs stay in shared memory until the end:
                esh[j] = al;                           // a global store pending at a cluster barrier
                dsh[j] = xg[j];                        // costs ~1200 cycles there
            }
        } else {
            constexpr int MV_ROWS = (TC_THREADS - 32) / NCH;
            for (int rb = 0; rb < nr; rb += MV_ROWS) {
                const int r = rb + tid / NCH, ch = tid - (tid / NCH) * NCH;
                double acc = 0.0, acc2 = 0.0;             // two chains: FP64 latency bounds this
                if (r < nr) {
                    const double* row = Srow + (li0 + r) * k;
                    int c = c0 + 1 + ch;
                    for (; c + NCH < k; c += 2 * NCH) {
                        acc = fma(row[c], xg[c], acc);
                        acc2 = fma(row[c + NCH], xg[c + NCH], acc2);
                    }
                    if (c < k) acc = fma(row[c], xg[c], acc);
                }
                acc += acc2;
                for (int o = NCH / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (ch == 0 && r < nr) qloc[r] = acc;
            }
        }
        __syncthreads();
        const double t_j = sc[0], v0 = sc[2];
        for (int c = c0 + tid; c < k; c += TC_THREADS)
            vl[c] = (t_j == 0.0) ? 0.0 : (c == c0 ? v0 : xg[c]);
        if (c0 % C == rank)                            // the owner's copy of row c0 before the update
            for (int c = c0 + tid; c < k; c += TC_THREADS) nrow[par][c] = Srow[(c0 / C) * k + c];
        if (warp == 0) {                               // nr <= 32: the owned rows are warp 0's lanes
            double s3 = 0.0;
            if (lane < nr) {
                const int li = li0 + lane, i = rank + li * C;
                const double vi = (t_j == 0.0) ? 0.0 : (i == c0 ? v0 : xg[i]);
                const double pi = t_j * fma(Srow[li * k + c0], v0, qloc[lane]);
                pown[par][li] = pi;
                s3 = pi * vi;
                Srow[li * k + j] = vi;                 // the reflector: column j of the row is dead now
            }
            s3 = warp_sum(s3);
            if (lane == 0) pvl[par] = s3;
        }
        cl.sync();
        // ---- C: p and the pivot row copy from their owners, w = p - (tau/2)(p^T v) v, then the
        // rank-2 update of the owned rows and of the copy (step j+1's pivot row)
        {
            const double* nsrc = cl.map_shared_rank(&nrow[par][0], c0 % C);
            for (int c = c0 + tid; c < k; c += TC_THREADS) {
                xn[c] = nsrc[c];
                if (t_j != 0.0) pg[c] = cl.map_shared_rank(&pown[par][0], c % C)[c / C];
            }
        }
        if (t_j != 0.0 && warp == 0) {
            const double t2 = warp_sum(lane < C ? *cl.map_shared_rank(&pvl[par], lane) : 0.0);
            if (lane == 0) sc[3] = 0.5 * t_j * t2;
        }
        __syncthreads();
        if (t_j != 0.0) {
            const double Kc = sc[3];
            for (int c = c0 + tid; c < k; c += TC_THREADS) wl[c] = pg[c] - Kc * vl[c];
            __syncthreads();
            // a warp per owned row, lanes along the columns; the operands are put in (lo, hi)
            // order by selects
            for (int r = warp; r < nr; r += TC_THREADS / 32) {
                const int li = li0 + r, i = rank + li * C;
                const double vi = vl[i], wi = wl[i];
                double* row = Srow + li * k;
                for (int c = c0 + lane; c < k; c += 32) {
                    const double vc = vl[c], wc = wl[c];
                    const bool up = c >= i;
                    const double x1 = up ? vi : vc, y1 = up ? wc : wi;
                    const double x2 = up ? wi : wc, y2 = up ? vc : vi;
                    row[c] = fma(-x1, y1, fma(-x2, y2, row[c]));
                }
            }
            // the next pivot row: row c0 updated exactly as its owner updates it (c >= c0 = i)
            const double vi = vl[c0], wi = wl[c0];
            for (int c = c0 + tid; c < k; c += TC_THREADS) xg[c] = fma(-vi, wl[c], fma(-wi, vl[c], xn[c]));
        } else {
            for (int c = c0 + tid; c < k; c += TC_THREADS) xg[c] = xn[c];
        }
        __syncthreads();
    }
    // ---- outputs: reflectors of the owned rows (A(i, j) = v_i of step j, j < min(i, k - 2)),
    // d for the owned rows, e and tau (every block holds them; block 0 writes)
    for (int li = warp; li < nloc; li += TC_THREADS / 32) {
        const int i = rank + li * C;
        const int jmax = min(i, k - 2);
        for (int j = lane; j < jmax; j += 32) A[(long long)j * lda + i] = Srow[li * k + j];
    }
    for (int j = rank + tid * C; j + 2 < k; j += TC_THREADS * C) d[j] = dsh[j];
    if (rank == 0)
        for (int j = tid; j + 2 < k; j += TC_THREADS) {
            e[j] = esh[j];
            tau[j] = tsh[j];
        }
    if (tid == 0) {
        if (k >= 2) {
            if ((k - 2) % C == rank) d[k - 2] = Srow[((k - 2) / C) * k + (k - 2)];
            if ((k - 1) % C == rank) {
                d[k - 1] = Srow[((k - 1) / C) * k + (k - 1)];
                e[k - 2] = Srow[((k - 1) / C) * k + (k - 2)];
            }
            if (rank == 0) tau[k - 2] = 0.0;
        } else if (k == 1 && rank == 0) {
            d[0] = Srow[0];
        }
    }
    cl.sync();                     // no block leaves while a peer could still address its memory
}

// ------------------------------------------------------------------ pivoted Cholesky
// Pivoted Cholesky P^T G P = Lt Lt^T of the k x k Gram G (diagonal pivoting; rank revealing
// for a PSD Gram Y^T Y).  Stops at the first pivot <= tol max(diag G), or <= 0, or <= the
// absolute floor floor_rel d0_ref (the numerical rank m); without pivoting a stop raises
// `fail`.  Output: Lt directly, slot u holding the row chosen at step u (Lt(u, s) at
// L[s ldl + u]); perm[u] the original index of slot u for every slot (rows never chosen take the
// slots m.. in increasing index); dm_out = m, kx_out = k; d0_out = max(diag G) if given.
// A near-identity Gram G = I + E (the last CholeskyQR pass, whose input is orthonormal to
// rounding) with ||E||_F^2 <= 1e-16 takes the factor I + F, F = strict_lower(E) + diag(E)/2:
// (I + F)(I + F)^T = G + F F^T and ||F F^T||_F <= ||E||_F^2, far below the factorisation's own
// rounding (~k u); no pivot is needed (every diagonal is 1 +- 1e-8).  Its inverse is written to
// W directly (the layout of the triangular inverse) and near_out[b] = 1.
// Right-looking over the cluster: block `rank` keeps, for its rows i = rank + li C, the current
// Schur complement row S(i, :) (ld k), the computed L(i, 0..t) (ld k) and the Schur diagonal.
// Step t (one cluster barrier):
//   pick the pivot q from the C candidates gathered at the last barrier (diagonal bits as the
//   key, ties to the smaller index; the same choice in every block);
//   apply step t-1's rank-1 update S(i, j) -= L(i, t-1) L(j, t-1) to the owned active rows over
//   the active columns (L(:, t-1) was gathered at the last barrier);
//   L(i, t) = S(i, q) / sqrt(d_q), d_i -= L(i, t)^2 for the owned active rows;
//   send the owned entries of L(:, t) and the block's best row for step t+1 to every block;
//   cluster barrier.
// Every block sends about (k - t) / C values a step and receives k - t: no block serves the
// others (a left-looking form has every block read the pivot row from its one owner).  Both
// buffers alternate by step parity: a block writes step t+1's data only after passing step t's
// barrier, and step t+2's after step t+1's, when every reader of step t's data is done.
template <int C>
__global__ void __launch_bounds__(TC_THREADS) k_chol_cluster(ModeMap mm, const double* G, long long gstride, int ldg,
                                                             const int* dk, int* kx_out, double* L, long long lstride,
                                                             int ldl, int* perm, int pstride, int* dm_out, int* fail,
                                                             int pivot, double tol, double* d0_out,
                                                             const double* d0_ref, double floor_rel, double* W,
                                                             long long wstride, int ldw, int* near_out)
{
    constexpr int ROWS = (KMAX + C - 1) / C;
    static_assert(ROWS <= 32, "row split");
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int b = mm.m[blockIdx.y];
    const int k = dk[b];
    G += b * gstride;
    L += b * lstride;
    W += b * wstride;
    perm += b * pstride;
    extern __shared__ double dyn[];
    double* Srow = dyn;                                    // ROWS x k
    double* Lrow = dyn + (size_t)ROWS * k;                 // ROWS x k
    __shared__ double colbuf[2][KMAX];
    __shared__ double dsh[32];
    __shared__ int act[32], pos[32], slot[32];
    __shared__ int gact[KMAX], gpos[KMAX];
    __shared__ long long ckey[2][C];
    __shared__ int cidx[2][C];
    __shared__ double cdp[2][C], cnear[C];
    __shared__ int pivs[KMAX];
    __shared__ unsigned char chosen[KMAX];
    __shared__ double red[TC_THREADS / 32];
    __shared__ double s_rp;
    __shared__ int s_q, s_stop, s_nact, s_gna;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nloc = rank < k ? (k - rank + C - 1) / C : 0;
    // row i of G = column i (G is symmetric)
    for (int li = warp; li < nloc; li += TC_THREADS / 32) {
        const int i = rank + li * C;
        for (int c = lane; c < k; c += 32) Srow[li * k + c] = G[(long long)i * ldg + c];
    }
    if (tid < 32) {
        act[tid] = tid;
        pos[tid] = tid;
        slot[tid] = -1;
    }
    for (int i = tid; i < k; i += TC_THREADS) {
        chosen[i] = 0;
        gact[i] = i;
        gpos[i] = i;
    }
    if (tid == 0) {
        s_nact = nloc;
        s_gna = k;
    }
    __syncthreads();
    if (tid < nloc) dsh[tid] = Srow[tid * k + rank + tid * C];
    // largest diagonal of G (every block reads all of it: k values)
    double dmx = 0.0;
    for (int i = tid; i < k; i += TC_THREADS) dmx = fmax(dmx, G[(long long)i * ldg + i]);
    dmx = warp_max(dmx);
    if (lane == 0) red[warp] = dmx;
    __syncthreads();
    double d0max = 0.0;
    for (int w = 0; w < TC_THREADS / 32; ++w) d0max = fmax(d0max, red[w]);
    if (d0_out && rank == 0 && tid == 0) d0_out[b] = d0max;
    const double dfloor = d0_ref ? floor_rel * d0_ref[b] : 0.0;
    // near-identity shortcut: ||G - I||_F^2 from the owned rows, summed over the blocks in
    // rank order
    const bool try_near = dfloor < 0.5 && tol * d0max < 0.5;
    if (try_near) {
        double s = 0.0;
        for (int li = warp; li < nloc; li += TC_THREADS / 32) {
            const int i = rank + li * C;
            for (int c = lane; c < k; c += 32) {
                const double g = Srow[li * k + c];
                const double ev = (c == i) ? g - 1.0 : g;
                s = fma(ev, ev, s);
            }
        }
        s = warp_sum(s);
        __syncthreads();
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (tid < C) {
            double t = 0.0;
            for (int w = 0; w < TC_THREADS / 32; ++w) t += red[w];
            cl.map_shared_rank(cnear, tid)[rank] = t;
        }
    }
    cl.sync();                     // all blocks loaded (and near-identity parts exchanged)
    if (try_near) {
        double s = 0.0;
        for (int r = 0; r < C; ++r) s += cnear[r];
        if (s <= 1e-16) {
            // the inverse directly, in the layout of the triangular inverse (W(perm[j], t) =
            // Lt^{-1}(t, j), perm = identity): Lt^{-1} = I - F to first order (error ||F||^2),
            // so W(j, t) = -G(t, j) for t > j, 1 - (G(j, j) - 1)/2 on the diagonal, 0 below.
            // W may share G's buffer: every block read its rows before the barrier above.
            for (int li = warp; li < nloc; li += TC_THREADS / 32) {
                const int j = rank + li * C;
                for (int t = lane; t < k; t += 32) {
                    const double g = Srow[li * k + t];
                    W[(long long)t * ldw + j] = t < j ? 0.0 : (t == j ? fma(-0.5, g - 1.0, 1.0) : -g);
                }
            }
            if (rank == 0) {
                for (int t = tid; t < k; t += TC_THREADS) perm[t] = t;
                if (tid == 0) {
                    dm_out[b] = k;
                    kx_out[b] = k;
                    if (near_out) near_out[b] = 1;
                }
            }
            cl.sync();
            return;
        }
    }
    // this block's best active row for a step, sent to every block (warp 0)
    auto send_candidate = [&](int par) {
        const int na = s_nact;
        long long key = LLONG_MIN;
        int idx = INT_MAX;
        double dv = 0.0;
        if (lane < na) {
            const int li = act[lane];
            dv = dsh[li];
            const long long bits = __double_as_longlong(dv);
            key = pivot ? (bits >= 0 ? bits : -1) : -1;   // unpivoted: every key ties, the index decides
            idx = rank + li * C;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
            const double d2 = __shfl_xor_sync(0xffffffffu, dv, o);
            if (k2 > key || (k2 == key && i2 < idx)) {
                key = k2;
                idx = i2;
                dv = d2;
            }
        }
        if (lane < C) {
            cl.map_shared_rank(&ckey[par][0], lane)[rank] = key;
            cl.map_shared_rank(&cidx[par][0], lane)[rank] = idx;
            cl.map_shared_rank(&cdp[par][0], lane)[rank] = dv;
        }
    };
    if (warp == 0) send_candidate(0);
    cl.sync();
    int m = k;
    for (int t = 0; t < k; ++t) {
        const int par = t & 1;
        // ---- the pivot: the best of the C candidates (a shuffle tree in warp 0: the same
        // maximum, ties to the smaller index, in any order)
        if (warp == 0) {
            long long kr = LLONG_MIN;
            int ir = INT_MAX;
            double dr = 0.0;
            if (lane < C) {
                kr = ckey[par][lane];
                ir = cidx[par][lane];
                dr = cdp[par][lane];
            }
            for (int o = 16; o > 0; o >>= 1) {
                const long long k2 = __shfl_xor_sync(0xffffffffu, kr, o);
                const int i2 = __shfl_xor_sync(0xffffffffu, ir, o);
                const double d2 = __shfl_xor_sync(0xffffffffu, dr, o);
                if (k2 > kr || (k2 == kr && i2 < ir)) {
                    kr = k2;
                    ir = i2;
                    dr = d2;
                }
            }
            if (lane == 0) {
                const int q = ir;
                const double dp = dr;
                const bool stop = q >= k || !(dp > tol * d0max) || !(dp > 0.0) || !(dp > dfloor);
                s_stop = stop;
                s_q = q;
                if (!stop) {
                    const double rp = fast_rsqrt(dp);      // one short chain instead of sqrt, then 1 / x
                    s_rp = rp;
                    pivs[t] = q;
                    chosen[q] = 1;
                    if (q % C == rank) {               // the owner: L(q, t), and q leaves the active rows
                        const int lq_ = q / C;
                        Lrow[lq_ * k + t] = dp * rp;
                        slot[lq_] = t;
                        const int p0 = pos[lq_], last = act[s_nact - 1];
                        act[p0] = last;
                        pos[last] = p0;
                        s_nact = s_nact - 1;
                    }
                }
            }
        }
        __syncthreads();
        if (s_stop) {
            if (!pivot && tid == 0 && fail && rank == 0) fail[b] = 1;
            m = t;
            break;
        }
        const int q = s_q;
        const double rp = s_rp;
        const int na = s_nact, gna = s_gna;
        // ---- step t-1's update of the owned active rows over the active columns (q still
        // among them: its column is read next)
        if (t > 0) {
            const double* lc = &colbuf[par ^ 1][0];
            for (int r = warp; r < na; r += TC_THREADS / 32) {
                const int li = act[r];
                const double lit = Lrow[li * k + t - 1];
                double* row = Srow + li * k;
                for (int u = lane; u < gna; u += 32) {
                    const int j = gact[u];
                    row[j] = fma(-lit, lc[j], row[j]);
                }
            }
            __syncthreads();
        }
        // ---- column t of the owned active rows, the new Schur diagonal
        if (tid < na) {
            const int li = act[tid];
            const double lit = Srow[li * k + q] * rp;
            Lrow[li * k + t] = lit;
            dsh[li] = fma(-lit, lit, dsh[li]);
        }
        __syncthreads();
        // ---- send the owned entries of L(:, t) and the next candidate; q leaves the active columns
        if (tid < na * C) {
            const int r = tid / C, dst = tid - r * C;
            const int li = act[r];
            cl.map_shared_rank(&colbuf[par][0], dst)[rank + li * C] = Lrow[li * k + t];
        }
        if (warp == 0) send_candidate(par ^ 1);
        if (tid == 32) {
            const int p0 = gpos[q], last = gact[gna - 1];
            gact[p0] = last;
            gpos[last] = p0;
            s_gna = gna - 1;
        }
        cl.sync();
    }
    // ---- outputs: the chosen rows of Lt in slot order, the permutation, the counts
    for (int li = warp; li < nloc; li += TC_THREADS / 32) {
        const int u = slot[li];
        if (u < 0 || u >= m) continue;
        for (int s2 = lane; s2 <= u; s2 += 32) L[(long long)s2 * ldl + u] = Lrow[li * k + s2];
    }
    if (rank == 0) {
        for (int u = tid; u < m; u += TC_THREADS) perm[u] = pivs[u];
        __syncthreads();
        if (tid == 0) {
            int u = m;
            for (int i = 0; i < k; ++i)
                if (!chosen[i]) perm[u++] = i;
            dm_out[b] = m;
            kx_out[b] = k;
            if (near_out) near_out[b] = 0;
        }
    }
    cl.sync();                     // no block leaves while a peer could still write its memory
}

template <int C>
static int launch_tridiag_c(ModeMap mm, double* A, long long astride, int lda, const int* dk, double* d, double* e,
                            double* tau, int vstride, int nb, int kbound, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        const int smax = (int)(sizeof(double) * ((KMAX + C - 1) / C) * KMAX);
        if (cudaFuncSetAttribute(k_tridiag_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        if (C > 8 && cudaFuncSetAttribute(k_tridiag_cluster<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                         cudaSuccess)
            return RHOSVD_ERR_CUDA;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, nb, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = sizeof(double) * (size_t)((kbound + C - 1) / C) * (size_t)kbound;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_tridiag_cluster<C>, mm, A, astride, lda, dk, d, e, tau, vstride) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    count_launch();
    return 0;
}

template <int C>
static int launch_chol_c(ModeMap mm, const double* G, long long gstride, int ldg, const int* dk, int* kx_out, double* L,
                         long long lstride, int ldl, int* perm, int pstride, int* dm_out, int* fail, int pivot,
                         double tol, int nb, int kbound, double* d0_out, const double* d0_ref, double floor_rel,
                         double* W, long long wstride, int ldw, int* near_out, cudaStream_t st)
{
    constexpr int ROWS = (KMAX + C - 1) / C;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_chol_cluster<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(double) * 2 * ROWS * KMAX)) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        if (C > 8 &&
            cudaFuncSetAttribute(k_chol_cluster<C>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, nb, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = sizeof(double) * 2 * (size_t)ROWS * (size_t)kbound;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_chol_cluster<C>, mm, G, gstride, ldg, dk, kx_out, L, lstride, ldl, perm, pstride,
                           dm_out, fail, pivot, tol, d0_out, d0_ref, floor_rel, W, wstride, ldw, near_out) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    count_launch();
    return 0;
}

// Cluster width for a kernel: 16 if a 16-block cluster of its blocks (smem16 bytes of dynamic
// shared memory each) can be resident, else 8 (portable).  Decided once per kernel.
template <typename Kern>
static int query_width(Kern kern, size_t smem16, int& width)
{
    if (width == 0) {
        width = 8;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem16) == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(16, 1, 1);
            cfg.blockDim = dim3(TC_THREADS, 1, 1);
            cfg.dynamicSmemBytes = smem16;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 16;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) width = 16;
        }
        cudaGetLastError();        // a refused query leaves no sticky error behind
    }
    return width;
}

int launch_tridiag_cluster(ModeMap mm, double* A, long long astride, int lda, const int* dk, double* d, double* e,
                           double* tau, int vstride, int nb, int kbound, cudaStream_t st)
{
    if (kbound > KMAX) return RHOSVD_ERR_INVALID_ARG;
    static int width = 0;
    if (query_width(k_tridiag_cluster<16>, sizeof(double) * ((KMAX + 15) / 16) * KMAX, width) == 16)
        return launch_tridiag_c<16>(mm, A, astride, lda, dk, d, e, tau, vstride, nb, kbound, st);
    return launch_tridiag_c<8>(mm, A, astride, lda, dk, d, e, tau, vstride, nb, kbound, st);
}

}  // namespace rh

namespace rh {

int launch_chol_cluster(ModeMap mm, const double* G, long long gstride, int ldg, const int* dk, int* kx_out, double* L,
                        long long lstride, int ldl, int* perm, int pstride, int* dm_out, int* fail, int pivot,
                        double tol, int nb, int kbound, double* d0_out, const double* d0_ref, double floor_rel,
                        double* W, long long wstride, int ldw, int* near_out, cudaStream_t st)
{
    if (kbound > KMAX) return RHOSVD_ERR_INVALID_ARG;
    static int width = 0;
    if (query_width(k_chol_cluster<16>, sizeof(double) * 2 * ((KMAX + 15) / 16) * KMAX, width) == 16)
        return launch_chol_c<16>(mm, G, gstride, ldg, dk, kx_out, L, lstride, ldl, perm, pstride, dm_out, fail, pivot,
                                 tol, nb, kbound, d0_out, d0_ref, floor_rel, W, wstride, ldw, near_out, st);
    return launch_chol_c<8>(mm, G, gstride, ldg, dk, kx_out, L, lstride, ldl, perm, pstride, dm_out, fail, pivot, tol,
                            nb, kbound, d0_out, d0_ref, floor_rel, W, wstride, ldw, near_out, st);
}

}  // namespace rh

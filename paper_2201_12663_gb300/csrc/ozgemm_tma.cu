// ozgemm_tma.cu -- the digit-plane tcgen05 GEMM (arithmetic in ozgemm.cuh) as a warp-specialised
// pipeline fed by the Tensor Memory Accelerator.
//
// One CTA computes a 128 x NT tile of C.  K advances in stages of 16 (one tcgen05.mma K step)
// through a ring of STAGES shared-memory buffers.  Warp roles:
//   warp 0     producer: lane 0 loads every digit plane of the stage's A and B tiles onto the
//              stage's "full" mbarrier: tile-major planes by cp.async.bulk (one contiguous block),
//              row-major planes by cp.async.bulk.tensor (2D tensor maps over this GPU's memory, no
//              multicast);
//   warp 1     MMA issuer: lane 0 waits for a full stage, issues one tcgen05.mma (kind::f16, BF16
//              digits, FP32 accumulation in TMEM) per digit pair (s, t) with s + t <= GMAX into
//              the accumulator of group g = s + t, and commits the stage's "empty" barrier;
//   warps 2-9  epilogue: read accumulators back into double-float registers (tcgen05.ld) when
//              their exactness cadence requires it, then store C or the residual energy.
// Tiles are K-major with the 32-byte swizzle (8-row x 32-byte atoms, 256 B between 8-row groups),
// the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_32B and the MMA descriptors read.
//
// Accumulators (Plan<KIND>): the MMAs of one lane plane s against the stacked col planes t write
// the groups g = s + t into consecutive column blocks, so a stage costs one MMA per lane plane.
// Two buffers of every group's columns alternate by blocks of RBK stages: while the MMAs fill one,
// the epilogue reads the other back into double-float registers.  Every group stays exact in FP32
// over its block (Plan<KIND>::ok checks np 2^(2W) 16 RBK <= 2^24).
//
// The Khatri-Rao core (k_ozcore, below) has its own warp roles: its A operand is formed in shared
// memory by the worker warps instead of being copied.
//
// Every mbarrier wait is bounded.  On expiry the CTA stops producing, issuing and reading back,
// waits (bounded again) for its own copies and MMAs in flight, records RHOSVD_ERR_TIMEOUT in the
// batch's status word (or the library's, see oz_take_status), frees TMEM and returns.
#include "ozgemm.cuh"
#include <cuda.h>
#include <climits>
#include <mutex>

namespace rh {

// status word of this file's products launched without a caller status (see oz_take_status)
__device__ int g_oztma_status = 0;

int oztma_take_status(cudaStream_t st, int* out)
{
    int v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_oztma_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbolAsync(g_oztma_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
    }
    *out = v;
    return RHOSVD_OK;
}

namespace {

constexpr int TK = 16;                  // K per stage
constexpr int T_WARPS = 10;
constexpr int T_THREADS = 32 * T_WARPS;
constexpr int T_EPI0 = 2;               // first epilogue warp
constexpr int T_NEPI = 8;               // epilogue warps: two per TMEM lane quarter
constexpr int T_SMEM_MAX = 227 * 1024;

struct OzMaps {
    CUtensorMap a[3];
    CUtensorMap b[3];
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, 32-byte swizzle: start address, LBO unused (16 B), SBO = 256 B, version 1, layout 6
__device__ __forceinline__ uint64_t desc_sw32(uint32_t addr)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(256 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;
    return d;
}

__host__ __device__ constexpr uint32_t idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(su32(b)),
                 "r"(bytes) : "memory");
}

// bounded wait for the phase of the given parity; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity)
{
    uint32_t done = 0;
    for (long it = 0; it < (1L << 24) && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(su32(b)), "r"(parity) : "memory");
    }
    return done != 0;
}

// the same with a short sleep between polls, for waits that are usually long
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* b, uint32_t parity)
{
    uint32_t done = 0;
    for (long it = 0; it < (1L << 22) && !done; ++it) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done) : "r"(su32(b)), "r"(parity) : "memory");
        if (!done) __nanosleep(128);
    }
    return done != 0;
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                 ::"r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
                 : "memory");
}

// one contiguous global -> shared copy onto an mbarrier (16-byte aligned, a multiple of 16 bytes)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(su32(dst)), "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar)) : "memory");
}

// One 32-lane x 16-column TMEM load; several are issued before one tcgen05.wait::ld
__device__ __forceinline__ void tmem_ld16_issue(uint32_t addr, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// The epilogues' conversions, from the bits, without branches.  GB300 issues FP64 instructions
// (the conversions between FP32 and FP64 among them) at about two lanes a cycle per SM, and a
// dependent FP64 operation waits ~64 cycles (several hundred behind a busy FP64 pipe): the
// store epilogue keeps one FP64 add per output element, all of an item's adds independent of one
// another and free of branches, so that they issue back to back; the residual none (FP32
// double-float arithmetic); the rest is integer work.
//
// x 2^e as a double, exactly, for a finite FP32 x: the exponent is rebiased and the 23 fraction
// bits move to the top of FP64's 52; an FP32 subnormal m 2^-149 is normalised first (its leading
// bit p: 1.f 2^(p - 149)).  Zero, and a result below FP64's normal range, give +0.
__device__ __forceinline__ double f2d_scaled(float x, int e)
{
    const uint32_t b = __float_as_uint(x);
    const uint32_t fe = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    const int p = 31 - __clz((int)(m | 1u));
    const uint32_t f = fe ? m : ((m << (23 - p)) & 0x7fffffu);
    const int be = (fe ? (int)fe - 127 : p - 149) + e + 1023;
    const uint32_t h = (b & 0x80000000u) | ((uint32_t)be << 20) | (f >> 3);
    return ((b << 1) == 0u || be <= 0) ? 0.0 : __hiloint2double((int)h, (int)(f << 29));
}

// hi + lo += x, with the error of the high sum kept exactly (Knuth's two-sum) but the pair not
// renormalised: seven operations instead of nine, for the residual's short sums (K = r <= 256:
// at most two readback blocks of eight groups, 16 additions, so the low word's own rounding
// stays below 2^-40 of the largest partial sum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    const float l = lo + err;
    hi = s + l;
    lo = l - (hi - s);
}

__host__ __device__ constexpr int npairs(int SA, int SB, int g)
{
    int c = 0;
    for (int s = 1; s <= SA; ++s)
        if (g - s >= 1 && g - s <= SB) ++c;
    return c;
}

// Plans.  The CTA tile is 128 rows of the "lane" operand (on the TMEM lanes) by NT rows of the
// "col" operand.  Each stage issues one MMA per digit plane s of the lane operand, against the
// col operand's planes t = 1 .. T(s) stacked along N, into the consecutive TMEM columns of the
// groups g = s + 1 .. s + T(s) (group g at NT (g - 2)): the MMA's N is NT T(s), up to 256, so a
// stage costs SL instructions instead of one per digit pair.  The first MMA of a block (s = 1)
// spans every group's columns (a zero plane fills the stack where needed) and overwrites them.
// Two accumulator buffers of NG NT columns alternate by blocks of RBK stages: the MMAs of block
// b + 1 run while the epilogue reads block b back into double-float registers.
//   TK_F64  (7 x 7 digits of 7 bits, pairs s + t <= 9): lane = A, col = B, NT = 32, 8 groups;
//           a group of np <= 7 pairs sums np 2^14 16 RBK <= 2^24 over a block of 8 stages, so
//           every group is exact until it is read back.
//   TK_SIGN (the range sketch, 7 digits of U~ against +-1): lane = the sign plane (the problem's
//           B, tile-major, 128 sketch columns, written once per sketch by k_sign_planes), col =
//           the U~ planes (the problem's A, tile-major, 32 rows of x), one MMA of N = 224 a
//           stage, 7 exact groups of one pair each.
//   TK_SIGN5 (the range sketch with five digits of U~): as TK_SIGN, one MMA of N = 160 a K step,
//           5 exact groups.
//   TK_BF16 (one plane of arbitrary BF16 values): lane = A, col = B, NT = 64, one group.
enum TmaKind { TK_F64 = 0, TK_SIGN = 1, TK_BF16 = 2, TK_SIGN5 = 3 };

template <int KIND>
struct Plan {
    static constexpr int SL = KIND == TK_F64 ? OZ_S64 : 1;
    static constexpr int SC = KIND == TK_BF16 ? 1 : (KIND == TK_SIGN5 ? OZ_S_SKETCH5 : OZ_S64);
    static constexpr int NT = KIND == TK_BF16 ? 64 : 32;
    static constexpr int GMAX = KIND == TK_F64 ? 9 : (KIND == TK_SIGN ? 8 : (KIND == TK_SIGN5 ? OZ_S_SKETCH5 + 1 : 2));
    static constexpr int W = KIND == TK_BF16 ? 8 : OZ_W64;
    static constexpr int NG = GMAX - 1;
    static constexpr int ZP = NG > SC ? NG - SC : 0;     // zero planes after the stacked ones
    static constexpr int NCOL = NG * NT;
    static constexpr int RBK = KIND == TK_F64 ? 8 : 16;   // K steps of 16 a readback block
    // K steps a pipeline stage: one producer thread completes about one stage per 0.7 us whatever
    // its size, so the sketch kinds (no zero plane between the steps' stacked planes) take four
    // (36 or 44 KB stages) and the FP64-class kinds two (their per-step col copies, 72 KB stages)
    static constexpr int KSUB = KIND == TK_BF16 ? 1 : (KIND == TK_F64 ? 2 : 4);
    static constexpr int RBS = RBK / KSUB;              // stages a readback block
    static constexpr int T(int s) { return s == 1 ? NG : (SC < GMAX - s ? SC : GMAX - s); }
    static constexpr bool ok()
    {
        bool good = 2 * NCOL <= 512 && NT * T(1) <= 256 && RBK % KSUB == 0;
        for (int g = 2; g <= GMAX && KIND != TK_BF16; ++g)
            good = good && (long long)npairs(SL, SC, g) * (1 << (2 * W)) * 16 * RBK <= (1 << 24);
        return good;
    }
};

__device__ __forceinline__ int dimv(const int* d, int h) { return d ? *d : h; }

}  // namespace

// One work item of a persistent CTA: problem pb, K split, lane tile tx, col tile ty; decoded the
// same way by every warp.  An item with no work (a split beyond the device's split count, or a
// tile outside the problem's device-side extent) is skipped by all of them.
struct TmaItem {
    int pb, split, tx, ty;
    int M, N, kbase, nkt;
    bool live;
};

template <int NT, int BK>
__device__ __forceinline__ TmaItem tma_item(const OzBatch& batch, int w, int ntx, int nty, int nsplit_h, bool sign)
{
    TmaItem it;
    it.tx = w % ntx;
    w /= ntx;
    it.ty = w % nty;
    w /= nty;
    it.split = w % nsplit_h;
    it.pb = w / nsplit_h;
    const OzProblem& P = batch.p[it.pb];
    const int nsplit = P.dsplit ? max(1, min(*P.dsplit, nsplit_h)) : nsplit_h;
    it.M = dimv(P.dM, P.M);
    it.N = dimv(P.dN, P.N);
    const int Kall = dimv(P.dK, P.K);
    // this item's K range: whole 32-wide blocks, the last split takes the rest
    const int kspan = ((Kall + nsplit - 1) / nsplit + BK - 1) / BK * BK;
    it.kbase = min(Kall, it.split * kspan);
    const int K = min(Kall, it.kbase + kspan) - it.kbase;
    it.nkt = (K + TK - 1) / TK;
    const int laneExt = sign ? it.N : it.M, colExt = sign ? it.M : it.N;
    it.live = it.split < nsplit && it.tx * OZ_BM < laneExt && it.ty * NT < colExt;
    return it;
}

// A persistent CTA: grid.x CTAs walk the items w = blockIdx.x, blockIdx.x + gridDim.x, ... (ntx lane
// tiles x nty col tiles x splits x problems).  The stage ring, the block counter and the
// accumulator buffers run on across items, so one item's readback and store overlap the next
// item's copies and MMAs.
template <int KIND, int EPI, int STAGES>
__global__ void __launch_bounds__(T_THREADS, 1) k_oztma(OzBatch batch, const __grid_constant__ OzMaps maps, int ntx,
                                                        int nty)
{
    using PL = Plan<KIND>;
    constexpr int SL = PL::SL, SC = PL::SC, NT = PL::NT, W = PL::W, NG = PL::NG, NCOL = PL::NCOL;
    constexpr int KSUB = PL::KSUB, RBS = PL::RBS;
    constexpr bool SIGN = KIND == TK_SIGN || KIND == TK_SIGN5;
    constexpr int L_PLANE = OZ_BM * TK * 2;              // 4096 B: 128 rows x 32 B
    constexpr int C_PLANE = NT * TK * 2;
    constexpr int L_BYTES = SL * L_PLANE;                  // one K step of the lane operand
    constexpr int C_BYTES = (SC + PL::ZP) * C_PLANE;      // one K step of the stacked operand
    constexpr int STAGE = (KSUB * (L_BYTES + C_BYTES) + 1023) / 1024 * 1024;
    constexpr int NC = NT / 2;                            // columns per epilogue warp
    constexpr int GB = NG < 4 ? NG : (EPI == OZ_EPI_RESID ? 2 : 4);   // groups a readback wait
    static_assert(PL::ok(), "plan: TMEM, MMA width or exactness");
    static_assert(NC % 16 == 0, "16-column TMEM loads");
    static_assert(STAGES * STAGE + 2048 <= T_SMEM_MAX, "shared memory");

    const int nsplit_h = batch.nsplit > 1 ? batch.nsplit : 1;
    const int nitems = ntx * nty * nsplit_h * batch.nbatch;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    extern __shared__ __align__(1024) unsigned char tsm[];
    unsigned char* stages = (unsigned char*)(((uintptr_t)tsm + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], buf_full[2], buf_free[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail, s_efail;
    __shared__ double red[T_NEPI];
    __shared__ int s_ec[T_NEPI][NC];     // the epilogue warps' column exponents of the current item

    // the zero planes of every stage (never written by the copies)
    if (PL::ZP > 0) {
        for (int s = 0; s < STAGES; ++s)
            for (int h = 0; h < KSUB; ++h) {
                uint32_t* z = (uint32_t*)(stages + s * STAGE + KSUB * L_BYTES + h * C_BYTES + SC * C_PLANE);
                for (int e = tid; e < PL::ZP * C_PLANE / 4; e += T_THREADS) z[e] = 0u;
            }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
    }
    if (tid == 32) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&buf_full[b], 1);
            mbar_init(&buf_free[b], T_NEPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
        s_efail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    volatile int* fail = &s_fail;

    if (warp == 0) {
        // ---------------------------------------------------------------- producer
        // lane 0 waits and decides; the decision is broadcast so that the warp stays converged
        int gs = 0;                         // stages issued so far (all items)
        for (int w = blockIdx.x; w < nitems && !*fail; w += gridDim.x) {
            const TmaItem it = tma_item<NT, OZ_BK>(batch, w, ntx, nty, nsplit_h, SIGN);
            if (!it.live) continue;
            const OzProblem& P = batch.p[it.pb];
            const OzPlanes& LP = SIGN ? P.B : P.A;
            const OzPlanes& CP = SIGN ? P.A : P.B;
            const int rowsL = LP.pstride > 0 ? (int)(LP.pstride / LP.ld) : 0;
            const int rowsC = CP.pstride > 0 ? (int)(CP.pstride / CP.ld) : 0;
            const int i0 = it.tx * OZ_BM, j0 = it.ty * NT;
            const int nst = (it.nkt + KSUB - 1) / KSUB;    // stages of the item (KSUB K steps each)
            bool stop = false;
            for (int kt = 0; kt < nst; ++kt, ++gs) {
                const int s = gs % STAGES;
                int go = 0;
                if (lane == 0) {
                    go = *fail ? 0 : 1;
                    if (go && gs >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((gs / STAGES) - 1) & 1))) {
                        *fail = 1;
                        go = 0;
                    }
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    stop = true;
                    break;
                }
                unsigned char* sL = stages + s * STAGE;
                unsigned char* sC = sL + KSUB * L_BYTES;
                const int k0 = it.kbase + kt * TK * KSUB;
                const int kk = min(KSUB, it.nkt - kt * KSUB);   // K steps in this stage
                if (lane == 0) {
                    mbar_expect_tx(&full[s], (uint32_t)kk * (L_BYTES + SC * C_PLANE));
                    if (LP.tiles_k > 0) {
                        // tile-major lane operand: the stage's kk x SL plane tiles are one contiguous
                        // block (consecutive k tiles of a row tile are adjacent)
                        const uint16_t* src = LP.base + ((long long)it.tx * LP.tiles_k + (k0 >> 4)) * SL * 2048;
                        bulk_g2s(sL, src, kk * L_BYTES, &full[s]);
                    } else {
                        // (row-major operands only in kinds of one K step a stage: ozgemm_tma_supports)
#pragma unroll
                        for (int p = 0; p < SL; ++p) tma_2d(sL + p * L_PLANE, &maps.a[it.pb], k0, p * rowsL + i0, &full[s]);
                    }
                    if (CP.tiles_k > 0) {
                        // tile-major col operand (NT-row tiles): the stage's SC plane tiles, one block
                        const uint16_t* src = CP.base + ((long long)it.ty * CP.tiles_k + (k0 >> 4)) * SC * (NT * 16);
                        if (PL::ZP == 0) {
                            bulk_g2s(sC, src, kk * SC * C_PLANE, &full[s]);
                        } else {
                            // a zero plane follows each K step's stacked planes: one copy a step
                            for (int h = 0; h < kk; ++h)
                                bulk_g2s(sC + h * C_BYTES, src + (long long)h * SC * (NT * 16), SC * C_PLANE, &full[s]);
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < SC; ++p) tma_2d(sC + p * C_PLANE, &maps.b[it.pb], k0, p * rowsC + j0, &full[s]);
                    }
                }
                __syncwarp();
            }
            if (stop) break;
        }
        if (*fail && lane == 0) {
            // copies in flight land before the CTA's shared memory goes away
            for (int g = max(0, gs - STAGES); g < gs; ++g) mbar_wait(&full[g % STAGES], (uint32_t)((g / STAGES) & 1));
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int gs = 0, gb = 0, last = -1;     // stages and blocks issued so far (all items)
            for (int w = blockIdx.x; w < nitems && !*fail; w += gridDim.x) {
                const TmaItem it = tma_item<NT, OZ_BK>(batch, w, ntx, nty, nsplit_h, SIGN);
                if (!it.live) continue;
                const int nst = (it.nkt + KSUB - 1) / KSUB;
                for (int kt = 0; kt < nst; ++kt, ++gs) {
                    if (*fail) break;
                    const int s = gs % STAGES;
                    const bool first = kt % RBS == 0;
                    const uint32_t buf = tmem + (uint32_t)((gb & 1) * NCOL);
                    // the block's buffer was read back by the epilogue two blocks ago
                    if (first && gb >= 2 && !mbar_wait(&buf_free[gb & 1], (uint32_t)(((gb >> 1) - 1) & 1))) {
                        *fail = 1;
                        break;
                    }
                    if (!mbar_wait(&full[s], (uint32_t)((gs / STAGES) & 1))) {
                        *fail = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t lBase = su32(stages + s * STAGE);
                    const int kk = min(KSUB, it.nkt - kt * KSUB);
#pragma unroll
                    for (int h = 0; h < KSUB; ++h) {
                        if (h >= kk) break;
                        const uint64_t dL0 = desc_sw32(lBase + (uint32_t)(h * L_BYTES));
                        const uint64_t dC0 = desc_sw32(lBase + (uint32_t)(KSUB * L_BYTES + h * C_BYTES));
#pragma unroll
                        for (int sp = 1; sp <= SL; ++sp) {
                            const uint32_t idesc = idesc_bf16(NT * PL::T(sp));
                            mma_f16(buf + (uint32_t)(NT * (sp - 1)), dL0 + (uint64_t)(((sp - 1) * L_PLANE) >> 4), dC0,
                                    idesc, (first && h == 0 && sp == 1) ? 0u : 1u);
                        }
                    }
                    mma_commit(&empty[s]);      // also tracks this stage's MMAs for the failure path
                    last = gs;
                    if (kt % RBS == RBS - 1 || kt + 1 == nst) {
                        mma_commit(&buf_full[gb & 1]);
                        ++gb;
                    }
                }
            }
            if (*fail && last >= 0) mbar_wait(&empty[last % STAGES], (uint32_t)((last / STAGES) & 1));
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- epilogue
        const int e = warp - T_EPI0;
        const int q = warp & 3;                  // TMEM lane quarter of this warp
        const int hcol = e >> 2;                 // which half of the NT columns
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int gb = 0;                              // blocks read back so far (all items)
        for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
            const TmaItem it = tma_item<NT, OZ_BK>(batch, w, ntx, nty, nsplit_h, SIGN);
            const OzProblem& P = batch.p[it.pb];
            if (!it.live) {
                if (EPI == OZ_EPI_RESID && e == 0 && lane == 0 && it.split == 0) P.rpart[it.tx + ntx * it.ty] = 0.0;
                continue;
            }
            const int nblk = ((it.nkt + KSUB - 1) / KSUB + RBS - 1) / RBS;
            float hi[NC], lo[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) { hi[c] = 0.f; lo[c] = 0.f; }
            // the entries' scale exponents (and the residual's reference entries) are loaded before
            // the item's readbacks, all at once, so that their latency passes while the item's
            // MMAs run instead of one load after another in the stores.  x = 2^(E - W) sum_s
            // plane_s: a product carries 2^(ea + eb - 2W), ea + eb = eL (this lane's operand row)
            // + the column's exponent, the same for the whole warp (kept in shared memory)
            const int lrow = it.tx * OZ_BM + q * 32 + lane;
            const int eL = SIGN ? W : ((lrow < it.M && P.A.exps) ? (int)P.A.exps[lrow] : P.A.exp0);
            {
                const OzPlanes& CPl = SIGN ? P.A : P.B;
                const int ccol = it.ty * NT + hcol * NC + lane;
                if (lane < NC) s_ec[e][lane] = (ccol < (SIGN ? it.M : it.N) && CPl.exps) ? (int)CPl.exps[ccol] : CPl.exp0;
                __syncwarp();
            }
            double rv[EPI == OZ_EPI_RESID ? NC : 1];
            if (EPI == OZ_EPI_RESID) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int ccol = it.ty * NT + hcol * NC + c;
                    const int row = SIGN ? ccol : lrow, col = SIGN ? lrow : ccol;
                    rv[c] = (row < it.M && col < it.N)
                                ? __ldg(P.ref + (long long)row * P.ref_rs + (long long)col * P.ref_cs)
                                : 0.0;
                }
            }
            for (int blk = 0; blk < nblk; ++blk, ++gb) {
                // lane 0 waits and decides for the warp (tcgen05.ld needs the whole warp converged)
                int go = 0;
                if (lane == 0) {
                    go = *fail ? 0 : 1;
                    if (go && !mbar_wait_sleep(&buf_full[gb & 1], (uint32_t)((gb >> 1) & 1))) {
                        *fail = 1;
                        go = 0;
                    }
                }
                if (!__shfl_sync(0xffffffffu, go, 0)) {
                    if (lane == 0) *(volatile int*)&s_efail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t buf = tmem + lane_base + (uint32_t)((gb & 1) * NCOL + hcol * NC);
                // up to four groups' loads in flight before one wait
#pragma unroll
                for (int g0 = 0; g0 < NG; g0 += GB) {
                    uint32_t v[GB][NC];
#pragma unroll
                    for (int g = 0; g < GB; ++g)
                        if (g0 + g < NG)
#pragma unroll
                            for (int c = 0; c < NC; c += 16) tmem_ld16_issue(buf + (uint32_t)((g0 + g) * NT + c), &v[g][c]);
                    tmem_ld_wait();
#pragma unroll
                    for (int g = 0; g < GB; ++g) {
                        if (g0 + g >= NG) continue;
#pragma unroll
                        for (int j = 0; j < NC; ++j) {
                            const float x = __uint_as_float(v[g][j]);
                            // the item's first value starts the sum (two_sum from zero gives the same)
                            if (g0 + g == 0 && blk == 0) { hi[j] = x; lo[j] = 0.f; }
                            else if (EPI == OZ_EPI_RESID) two_sum_acc(hi[j], lo[j], x);
                            else two_sum(hi[j], lo[j], x);
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                // the MMA issuer waits for this before the buffer's next block (extra arrivals
                // after the last block are never waited for)
                if (lane == 0) mbar_arrive(&buf_free[gb & 1]);
            }
            // the epilogue warps decide together: a warp whose readback failed has set s_efail
            // before this barrier, and nothing else writes it
            asm volatile("bar.sync 1, %0;" ::"r"(T_NEPI * 32) : "memory");
            if (*(volatile int*)&s_efail) break;
            const int M = it.M, N = it.N;
            const int j0 = it.ty * NT;
            const int nsplit = P.dsplit ? max(1, min(*P.dsplit, nsplit_h)) : nsplit_h;
            double* const Cout = nsplit > 1 ? P.Cpart + it.split * P.split_stride : P.C;
            const long long ccs = P.ccs < 0 ? (long long)M : P.ccs;
            const long long crs = P.crs < 0 ? (long long)N : P.crs;
            float e2f = 0.f;
            if (EPI == OZ_EPI_STORE) {
                // (hi + lo) 2^se: both parts scaled exactly, one FP64 add; the adds of all NC
                // entries first, then the stores, the bounds as predicates
                double tv[NC];
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int se = eL + s_ec[e][c] - 2 * W;
                    tv[c] = f2d_scaled(hi[c], se) + f2d_scaled(lo[c], se);
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int ccol = j0 + hcol * NC + c;              // col operand row
                    const int row = SIGN ? ccol : lrow, col = SIGN ? lrow : ccol;
                    if (row < M && col < N) Cout[(long long)row * crs + (long long)col * ccs] = tv[c];
                }
            } else {
                // d = ref - (hi + lo) 2^se in FP32 arithmetic: ref = rh + rl, the cancelling part
                // rh - hi 2^se exactly by two-sum (the scaling is exact), the small parts added to
                // its error.  |d - exact| <= 2^-24 |d| + ~2^-46 |ref|: the residual energy keeps
                // 2^-22 of itself wherever it matters (entries of eps |ref| and more), and the
                // entries' absolute errors add at most 2^-92 ||ref||^2 to it.  A scale or a part
                // below FP32's normal range only drops a term below 2^-126.
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const int ccol = j0 + hcol * NC + c;              // col operand row
                    const int row = SIGN ? ccol : lrow, col = SIGN ? lrow : ccol;
                    const float sf = pow2f(eL + s_ec[e][c] - 2 * W);
                    const float h = __fmul_rn(hi[c], sf), l = __fmul_rn(lo[c], sf);
                    float rh, rl;
                    split_f64(rv[EPI == OZ_EPI_RESID ? c : 0], rh, rl);
                    const float s1 = __fsub_rn(rh, h);
                    const float bp = __fsub_rn(s1, rh);
                    const float e1 = __fadd_rn(__fsub_rn(rh, __fsub_rn(s1, bp)), __fsub_rn(-h, bp));
                    const float d = __fadd_rn(s1, __fadd_rn(e1, __fsub_rn(rl, l)));
                    e2f = (row < M && col < N) ? fmaf(d, d, e2f) : e2f;
                }
            }
            if (EPI == OZ_EPI_RESID) {
                // the warp's sum in FP32 (32 partial sums of 16 squares), one conversion
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) e2f += __shfl_xor_sync(0xffffffffu, e2f, o);
                if (lane == 0) red[e] = (double)e2f;
                asm volatile("bar.sync 1, %0;" ::"r"(T_NEPI * 32) : "memory");
                if (e == 0 && lane == 0) {
                    double t = 0.0;
#pragma unroll
                    for (int w2 = 0; w2 < T_NEPI; ++w2) t += red[w2];
                    P.rpart[it.tx + ntx * it.ty] = t;
                }
                // red[] is rewritten only after every warp has read this item's sum
                asm volatile("bar.sync 1, %0;" ::"r"(T_NEPI * 32) : "memory");
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*fail && tid == 0) atomicCAS(batch.err ? batch.err : &g_oztma_status, 0, RHOSVD_ERR_TIMEOUT);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------- the Khatri-Rao core
// beta(i1, (j, m)) = sum_nu V1'(i1, nu) V2(j, nu) V3(m, nu) with V1' = V1 diag(xi'): C = A B^T
// with A the generated Khatri-Rao operand (row j + r2 m, k = nu) and B the digit planes of V1'.
// A CTA owns 128 rows of A (the TMEM lanes) and 160 rows of B (every r1 <= 160 at once); K runs
// in stages of 16 through a ring of four shared-memory stages.  Warp roles:
//   warp 0       MMA issuer: lane 0 issues, per stage, one tcgen05.mma of N = 160 per digit pair
//                (s, t) with s + t <= 5 into the accumulator of its group;
//   warps 1-16   workers: each thread forms 4 entries of A a stage (one row, 4 consecutive nu)
//                from the FP32 pairs of V2 and V3 and writes their 4 digit planes into the stage;
//                worker 0 also issues the stage's one bulk copy of B (tile-major, 160-row tiles);
//                every 256 K they read the accumulators back into double-float sums (40 columns of
//                one TMEM lane quarter a warp: the high words in registers, the low words in
//                shared memory) and at the end store beta.
// Both operands have balanced digits (|d1| <= 256, the others <= 128).  Three accumulators of 160
// columns: the group g = 2 (products below 2^16: exact for 256 K), the group 3 (two pairs below
// 2^15 each: exact for 256 K) and the groups 4 and 5 together in FP32 (their sum is below 2^-16
// of the leading group's scale).  480 of the 512 TMEM columns, so there is no second buffer: the
// MMAs of a block wait until the workers have read the previous one back, while the next stages
// are already formed.
namespace {

constexpr int C_NT = OZ_CORE_NT;               // B rows (r1) a CTA
constexpr int C_SK = 16;                       // K a stage (one MMA K step)
constexpr int C_STAGES = 4;
constexpr int C_WORK = 16;                     // worker warps
constexpr int C_THREADS = 32 * (1 + C_WORK);
constexpr int C_RBK = 16;                      // stages a readback block (256 K)
constexpr int C_A_PLANE = OZ_BM * C_SK * 2;    // one digit plane of A: 4096 B
constexpr int C_B_PLANE = C_NT * C_SK * 2;     // 5120 B
constexpr int C_A_BYTES = 4 * C_A_PLANE;
constexpr int C_B_BYTES = 4 * C_B_PLANE;
constexpr int C_STAGE = C_A_BYTES + C_B_BYTES;
constexpr int C_LO_BYTES = C_NT * OZ_BM * 4;   // low words of the double-float sums
constexpr int C_SMEM = C_STAGES * C_STAGE + C_LO_BYTES + 1024;
constexpr int C_COLS = C_NT / 4;               // output columns of a worker warp
static_assert(C_STAGE % 1024 == 0 && C_SMEM + 1024 <= T_SMEM_MAX, "core shared memory (and the static part)");
static_assert(3 * C_NT <= 512 && C_COLS % 8 == 0, "three accumulators in TMEM, 8-column loads");
// exactness over a block: group 2 (one pair below 2^16), group 3 (two pairs below 2^15)
static_assert(1LL * (1 << 16) * C_RBK * C_SK <= (1 << 24) && 2LL * (1 << 15) * C_RBK * C_SK <= (1 << 24),
              "core readback cadence");

// The four digit planes of one entry x = V2(j, nu) V3(m, nu) of the Khatri-Rao operand, row
// exponent E (|x| < 2^E), scale T = 2^(32 - E): F = round(x_hi T) + round(x_lo T) with x_hi the
// FP32 product of the heads and x_lo its error plus the cross terms (the tails' product, below
// 2^-46 of x, is dropped).  F is cut into balanced base-256 digits by rounding to multiples of
// 2^24, 2^16 and 2^8 (adding and subtracting 1.5 2^(23 + b) rounds an integer below 2^(22 + b)
// to a multiple of 2^b); every step is exact on integers below 2^24.  |d1| <= 256, |d2|, |d3|,
// |d4| <= 128; plane s holds d_s 2^(-8(s-1)), exact in BF16.
__device__ __forceinline__ void kr_digits(float2 a, float2 b, float T, float* v)
{
    const float ph = __fmul_rn(a.x, b.x);
    float pe = fmaf(a.x, b.x, -ph);
    pe = fmaf(a.x, b.y, fmaf(a.y, b.x, pe));
    const float yh = rintf(__fmul_rn(ph, T));
    const float yl = rintf(__fmul_rn(pe, T));
    const float t1 = __fsub_rn(__fadd_rn(yh, 0x1.8p47f), 0x1.8p47f);
    float r = __fadd_rn(__fsub_rn(yh, t1), yl);
    const float t2 = __fsub_rn(__fadd_rn(r, 0x1.8p39f), 0x1.8p39f);
    r = __fsub_rn(r, t2);
    const float t3 = __fsub_rn(__fadd_rn(r, 0x1.8p31f), 0x1.8p31f);
    r = __fsub_rn(r, t3);
    v[0] = __fmul_rn(t1, 0x1p-24f);
    v[1] = __fmul_rn(t2, 0x1p-24f);
    v[2] = __fmul_rn(t3, 0x1p-24f);
    v[3] = __fmul_rn(r, 0x1p-24f);
}

__device__ __forceinline__ void tmem_ld8_nowait(uint32_t addr, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
}

// row exponent of Khatri-Rao row i (j = i mod r2, m = i / r2)
__device__ __forceinline__ int kr_exp(const OzKR& kr, int i, int r2)
{
    return kr.e2 ? (int)kr.e2[i % r2] + (int)kr.e3[i / r2] : 0;
}

}  // namespace

__global__ void __launch_bounds__(C_THREADS, 1) k_ozcore(OzBatch batch)
{
    constexpr uint32_t IDESC = idesc_bf16(C_NT);
    const int nsplit_h = batch.nsplit > 1 ? batch.nsplit : 1;
    const int split = blockIdx.z % nsplit_h;
    const OzProblem& P = batch.p[blockIdx.z / nsplit_h];
    const int nsplit = P.dsplit ? max(1, min(*P.dsplit, nsplit_h)) : nsplit_h;
    if (split >= nsplit) return;
    const int r2 = *P.dNa;
    const int M = r2 * (*P.dNb);
    const int N = dimv(P.dN, P.N);
    const int Kall = dimv(P.dK, P.K);
    // this CTA's K range [kbase, kend): whole 32-wide pieces, the last split takes the rest
    const int kspan = ((Kall + nsplit - 1) / nsplit + OZ_BK - 1) / OZ_BK * OZ_BK;
    const int kbase = min(Kall, split * kspan);
    const int kend = min(Kall, kbase + kspan);
    double* const Cout = nsplit > 1 ? P.Cpart + split * P.split_stride : P.C;
    const int i0 = blockIdx.x * OZ_BM, j0 = blockIdx.y * C_NT;
    if (i0 >= M || j0 >= N) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkt = (kend - kbase + C_SK - 1) / C_SK;
    const int nblk = (nkt + C_RBK - 1) / C_RBK;

    extern __shared__ __align__(1024) unsigned char csm[];
    unsigned char* stages = (unsigned char*)(((uintptr_t)csm + 1023) & ~(uintptr_t)1023);
    float* const lo_s = reinterpret_cast<float*>(stages + C_STAGES * C_STAGE);   // [column][row]
    __shared__ __align__(8) uint64_t afull[C_STAGES], bfull[C_STAGES], empty[C_STAGES], acc_full, acc_free;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::);
    }
    if (tid == 32) {
        for (int s = 0; s < C_STAGES; ++s) {
            mbar_init(&afull[s], C_WORK);
            mbar_init(&bfull[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_free, C_WORK);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    volatile int* fail = &s_fail;
    int last = -1;          // MMA issuer: the stage committed last
    int issued_b = 0;       // worker 0: stages whose B copy was issued
    float hi[C_COLS];
    const int q = warp & 3;                 // TMEM lane quarter of a worker warp
    const int cg = (warp - 1) >> 2;         // its 40 output columns
    const int orow = q * 32 + lane;         // its output row in the tile

    if (warp == 0) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            for (int kt = 0; kt < nkt; ++kt) {
                if (*fail) break;
                const int s = kt % C_STAGES;
                const int blk = kt / C_RBK;
                const bool first = kt % C_RBK == 0;
                // the accumulators were read back after the previous block
                if (first && blk >= 1 && !mbar_wait(&acc_free, (uint32_t)((blk - 1) & 1))) {
                    *fail = 1;
                    break;
                }
                const uint32_t par = (uint32_t)((kt / C_STAGES) & 1);
                if (!mbar_wait(&bfull[s], par) || !mbar_wait(&afull[s], par)) {
                    *fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = su32(stages + s * C_STAGE);
                const uint64_t dA0 = desc_sw32(base), dB0 = desc_sw32(base + C_A_BYTES);
#pragma unroll
                for (int sa = 1; sa <= 4; ++sa) {
#pragma unroll
                    for (int tb = 1; tb <= 4; ++tb) {
                        if (sa + tb > 5) continue;
                        const int a = sa + tb - 2 < 2 ? sa + tb - 2 : 2;
                        // (1, 1), (1, 2), (1, 3) open the accumulators of groups 2, 3, 4-5
                        const bool reset = first && sa == 1 && tb <= 3;
                        mma_f16(tmem + (uint32_t)(a * C_NT), dA0 + (uint64_t)(((sa - 1) * C_A_PLANE) >> 4),
                                dB0 + (uint64_t)(((tb - 1) * C_B_PLANE) >> 4), IDESC, reset ? 0u : 1u);
                    }
                }
                mma_commit(&empty[s]);
                last = kt;
                if (kt % C_RBK == C_RBK - 1 || kt + 1 == nkt) mma_commit(&acc_full);
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------------- workers
        const int w = warp - 1;
#pragma unroll
        for (int c = 0; c < C_COLS; ++c) {
            hi[c] = 0.f;
            lo_s[(cg * C_COLS + c) * OZ_BM + orow] = 0.f;
        }
        // generation unit: row gr of the tile, k = 4 c4 .. 4 c4 + 3 of each stage; a warp covers 8
        // whole rows, so its digit stores fill 256 contiguous bytes of a plane
        const int gr = w * 8 + (lane >> 2), c4 = lane & 3;
        const int gi = i0 + gr;
        const bool live = gi < M;
        // the lanes' rows are consecutive: their V2 pairs are adjacent, their V3 pairs mostly one
        const float2* V2 = P.kr.V2p + (live ? gi % r2 : 0);
        const float2* V3 = P.kr.V3p + (live ? gi / r2 : 0);
        const long long ldp = P.kr.ldp;
        const float T = __int_as_float((127 + 32 - (live ? kr_exp(P.kr, gi, r2) : 0)) << 23);
        // 8 bytes (4 k) of row gr in the 32-byte swizzled plane tile
        const uint32_t a_off = (uint32_t)(gr * 32 + (((c4 >> 1) ^ ((gr >> 2) & 1)) << 4) + ((c4 & 1) << 3));

        // read block b back (whole warp; false once a wait has failed)
        auto readback = [&](int b) -> bool {
            int go = 0;
            if (lane == 0) {
                go = *fail ? 0 : 1;
                if (go && !mbar_wait_sleep(&acc_full, (uint32_t)(b & 1))) {
                    *fail = 1;
                    go = 0;
                }
            }
            if (!__shfl_sync(0xffffffffu, go, 0)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cg * C_COLS);
#pragma unroll
            for (int c = 0; c < C_COLS; c += 8) {
                uint32_t v[3][8];
                tmem_ld8_nowait(acc + (uint32_t)(2 * C_NT + c), v[2]);
                tmem_ld8_nowait(acc + (uint32_t)(C_NT + c), v[1]);
                tmem_ld8_nowait(acc + (uint32_t)c, v[0]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float* lp = lo_s + (cg * C_COLS + c + j) * OZ_BM + orow;
                    float l = *lp;
                    two_sum(hi[c + j], l, __uint_as_float(v[2][j]));
                    two_sum(hi[c + j], l, __uint_as_float(v[1][j]));
                    two_sum(hi[c + j], l, __uint_as_float(v[0][j]));
                    *lp = l;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0 && b + 1 < nblk) mbar_arrive(&acc_free);
            return true;
        };

        int rb = 0;                 // next block to read back
        for (int kt = 0; kt < nkt; ++kt) {
            // the MMAs of stage kt - C_STAGES (which frees this stage) follow block rb's readback
            if (rb < nblk && kt >= (rb + 1) * C_RBK + C_STAGES) {
                if (!readback(rb)) break;
                ++rb;
            }
            const int s = kt % C_STAGES;
            int go = 0;
            if (lane == 0) {
                go = *fail ? 0 : 1;
                if (go && kt >= C_STAGES && !mbar_wait(&empty[s], (uint32_t)(((kt / C_STAGES) - 1) & 1))) {
                    *fail = 1;
                    go = 0;
                }
            }
            if (!__shfl_sync(0xffffffffu, go, 0)) break;
            unsigned char* sA = stages + s * C_STAGE;
            const int k0 = kbase + kt * C_SK;
            if (w == 0 && lane == 0) {
                // the stage's B: one 16-wide k tile of the 160-row tile, contiguous
                const uint16_t* src = P.B.base + ((long long)(j0 / C_NT) * P.B.tiles_k + (k0 >> 4)) * 4 * (C_NT * C_SK);
                mbar_expect_tx(&bfull[s], (uint32_t)C_B_BYTES);
                bulk_g2s(sA + C_A_BYTES, src, (uint32_t)C_B_BYTES, &bfull[s]);
                issued_b = kt + 1;
            }
            const int kg = k0 + c4 * 4;
            uint32_t pk[4][2];
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {
                float v[2][4];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int k = kg + 2 * e2 + e;
                    float2 a = make_float2(0.f, 0.f), bb = a;
                    if (live && k < kend) {
                        a = __ldg(V2 + k * ldp);
                        bb = __ldg(V3 + k * ldp);
                    }
                    kr_digits(a, bb, T, v[e]);
                }
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    pk[p][e2] = __byte_perm(__float_as_uint(v[0][p]), __float_as_uint(v[1][p]), 0x7632);
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) *reinterpret_cast<uint2*>(sA + a_off + p * C_A_PLANE) = make_uint2(pk[p][0], pk[p][1]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&afull[s]);
        }
        while (rb < nblk && !*fail) {
            if (!readback(rb)) break;
            ++rb;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    const bool failed = *fail != 0;
    if (failed) {
        // what is still in flight lands before TMEM and shared memory go away
        if (tid == 0 && last >= 0) mbar_wait(&empty[last % C_STAGES], (uint32_t)((last / C_STAGES) & 1));
        if (tid == 32)
            for (int kt = max(0, issued_b - C_STAGES); kt < issued_b; ++kt)
                mbar_wait(&bfull[kt % C_STAGES], (uint32_t)((kt / C_STAGES) & 1));
        if (tid == 0) atomicCAS(batch.err ? batch.err : &g_oztma_status, 0, RHOSVD_ERR_TIMEOUT);
    } else if (warp > 0) {
        const int row = i0 + orow;
        if (row < M) {
            const int ea = kr_exp(P.kr, row, r2);
            const long long crs = P.crs < 0 ? (long long)N : P.crs;
            const long long ccs = P.ccs < 0 ? (long long)M : P.ccs;
#pragma unroll
            for (int c = 0; c < C_COLS; ++c) {
                const int col = j0 + cg * C_COLS + c;
                if (col >= N) continue;
                const int eb = P.B.exps ? (int)P.B.exps[col] : P.B.exp0;
                // planes carry x 2^(8 - E): the product's scale is 2^(ea + eb - 16)
                const int se = ea + eb - 16;
                const float lo = lo_s[(cg * C_COLS + c) * OZ_BM + orow];
                Cout[(long long)row * crs + (long long)col * ccs] = f2d_scaled(hi[c], se) + f2d_scaled(lo, se);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// streaming multiprocessors of the current device (the persistent kernels' CTA count)
int sm_count()
{
    static int cnt[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cnt[dev]) {
        int c = 0;
        if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = 1;
        cnt[dev] = c;
    }
    return cnt[dev];
}

// 2D map over S planes of `rows` rows each (ld elements a row, bf16 patterns): dims {ld, S rows},
// box {16, box_rows}, 32-byte swizzle, zero fill outside
bool plane_map(CUtensorMap* m, const OzPlanes& pl, int S, int rows, int box_rows)
{
    EncodeTiledFn enc = encoder();
    if (!enc || !pl.base || pl.ld <= 0 || pl.ld % 8 != 0 || rows <= 0) return false;
    if (((uintptr_t)pl.base) % 16 != 0) return false;
    if (S > 1 && pl.pstride != (long long)rows * pl.ld) return false;
    cuuint64_t dims[2] = {(cuuint64_t)pl.ld, (cuuint64_t)S * (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pl.ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)pl.base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KIND, int EPI>
int run_tma(const OzBatch& b, cudaStream_t st)
{
    using PL = Plan<KIND>;
    constexpr bool SIGN = KIND == TK_SIGN || KIND == TK_SIGN5;
    constexpr int L_BYTES = PL::SL * OZ_BM * TK * 2, C_PLANE = PL::NT * TK * 2;
    constexpr int STAGE = (PL::KSUB * (L_BYTES + (PL::SC + PL::ZP) * C_PLANE) + 1023) / 1024 * 1024;
    constexpr int ST_FIT = (T_SMEM_MAX - 4096) / STAGE;
    constexpr int STAGES = ST_FIT > 8 ? 8 : ST_FIT;
    static_assert(STAGES >= 2, "two stages at least");
    constexpr int SMEM = STAGES * STAGE + 1024;
    int Mh = 0, Nh = 0;
    for (int i = 0; i < b.nbatch; ++i) {
        Mh = max(Mh, b.p[i].M);
        Nh = max(Nh, b.p[i].N);
    }
    if (Mh <= 0 || Nh <= 0) return 0;
    OzMaps maps;
    memset(&maps, 0, sizeof(maps));
    for (int i = 0; i < b.nbatch; ++i) {
        const OzProblem& q = b.p[i];
        if (!SIGN && q.A.tiles_k <= 0) {
            const int ra = q.A.pstride > 0 ? (int)(q.A.pstride / (q.A.ld > 0 ? q.A.ld : 1)) : q.M;
            if (!plane_map(&maps.a[i], q.A, PL::SL, ra, OZ_BM)) return RHOSVD_ERR_INVALID_ARG;
        }
        const OzPlanes& cp = SIGN ? q.A : q.B;
        if (cp.tiles_k <= 0) {
            const int rc = cp.pstride > 0 ? (int)(cp.pstride / (cp.ld > 0 ? cp.ld : 1)) : (SIGN ? q.M : q.N);
            if (!plane_map(&maps.b[i], cp, PL::SC, rc, PL::NT)) return RHOSVD_ERR_INVALID_ARG;
        }
    }
    auto kern = k_oztma<KIND, EPI, STAGES>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        attr = true;
    }
    const int nsplit = b.nsplit > 1 ? b.nsplit : 1;
    if (nsplit > 1 && EPI != OZ_EPI_STORE) return RHOSVD_ERR_INVALID_ARG;
    const int laneExt = SIGN ? Nh : Mh, colExt = SIGN ? Mh : Nh;
    const int ntx = (laneExt + OZ_BM - 1) / OZ_BM, nty = (colExt + PL::NT - 1) / PL::NT;
    const long long nitems = (long long)ntx * nty * b.nbatch * nsplit;
    if (nitems > INT_MAX) return RHOSVD_ERR_INVALID_ARG;
    const int ncta = (int)(nitems < sm_count() ? nitems : sm_count());
    kern<<<ncta, T_THREADS, SMEM, st>>>(b, maps, ntx, nty);
    RH_CHECK_LAUNCH();
    return 0;
}

}  // namespace

namespace {

__global__ void k_selftest_bits(const double* x, const float* f, const int* e, float* rh, float* rl, double* fd,
                                float* p2, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        split_f64(x[i], rh[i], rl[i]);
        fd[i] = f2d_scaled(f[i], e[i]);
        p2[i] = pow2f(e[i]);
    }
}

}  // namespace

bool ozcore_tma_supports(const OzBatch& b)
{
    for (int i = 0; i < b.nbatch; ++i) {
        const OzProblem& q = b.p[i];
        if (!q.kr.V2p || !q.kr.V3p || !q.dNa || !q.dNb || !q.B.base || ((uintptr_t)q.B.base) % 16 != 0) return false;
        if (q.B.tiles_k <= 0 || q.B.tile_h != C_NT) return false;
    }
    return true;
}

int launch_ozcore_tma(const OzBatch& b, cudaStream_t st)
{
    int Mh = 0, Nh = 0;
    for (int i = 0; i < b.nbatch; ++i) {
        Mh = max(Mh, b.p[i].M);
        Nh = max(Nh, b.p[i].N);
    }
    if (Mh <= 0 || Nh <= 0) return 0;
    if (!ozcore_tma_supports(b)) return RHOSVD_ERR_INVALID_ARG;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_ozcore, cudaFuncAttributeMaxDynamicSharedMemorySize, C_SMEM) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        attr = true;
    }
    const int nsplit = b.nsplit > 1 ? b.nsplit : 1;
    dim3 grid((Mh + OZ_BM - 1) / OZ_BM, (Nh + C_NT - 1) / C_NT, b.nbatch * nsplit);
    k_ozcore<<<grid, C_THREADS, C_SMEM, st>>>(b);
    RH_CHECK_LAUNCH();
    return 0;
}

bool ozgemm_tma_supports(const OzBatch& b, OzKind kind)
{
    if (kind != OZ_F64_STORE && kind != OZ_F64_RESID && kind != OZ_SKETCH && kind != OZ_SKETCH5 && kind != OZ_BF16)
        return false;
    const bool sketch = kind == OZ_SKETCH || kind == OZ_SKETCH5;
    if (!encoder()) return false;
    const int S = kind == OZ_BF16 ? 1 : OZ_S64;
    const int nt = kind == OZ_BF16 ? Plan<TK_BF16>::NT : Plan<TK_F64>::NT;
    for (int i = 0; i < b.nbatch; ++i) {
        const OzProblem& q = b.p[i];
        // the operand on the TMEM lanes and the one stacked along N (the sketch swaps them)
        const OzPlanes* ops[2] = {sketch ? &q.B : &q.A, sketch ? &q.A : &q.B};
        for (int o = 0; o < 2; ++o) {
            const OzPlanes& pl = *ops[o];
            if (!pl.base || ((uintptr_t)pl.base) % 16 != 0) return false;
            if (pl.tiles_k > 0) {
                if (pl.tile_h != (o == 0 ? OZ_BM : nt)) return false;
                continue;
            }
            // the kinds of two K steps a stage read tile-major planes only (their row-major
            // tensor-map path would fetch one K step)
            if (kind != OZ_BF16) return false;
            if (pl.ld <= 0 || pl.ld % 8 != 0) return false;
            if (S > 1 && (pl.pstride <= 0 || pl.pstride % pl.ld != 0)) return false;
        }
    }
    return true;
}

// the residual partials one launch writes per problem (tiles of its grid)
long long ozgemm_tma_tiles(OzKind kind, int M, int N)
{
    const int nt = kind == OZ_BF16 ? Plan<TK_BF16>::NT : Plan<TK_F64>::NT;
    if (kind == OZ_SKETCH || kind == OZ_SKETCH5)
        return (long long)((N + OZ_BM - 1) / OZ_BM) * ((M + Plan<TK_SIGN>::NT - 1) / Plan<TK_SIGN>::NT);
    return (long long)((M + OZ_BM - 1) / OZ_BM) * ((N + nt - 1) / nt);
}

int launch_ozgemm_tma(const OzBatch& b, OzKind kind, cudaStream_t st)
{
    switch (kind) {
    case OZ_F64_STORE: return run_tma<TK_F64, OZ_EPI_STORE>(b, st);
    case OZ_F64_RESID: return run_tma<TK_F64, OZ_EPI_RESID>(b, st);
    case OZ_SKETCH: return run_tma<TK_SIGN, OZ_EPI_STORE>(b, st);
    case OZ_SKETCH5: return run_tma<TK_SIGN5, OZ_EPI_STORE>(b, st);
    case OZ_BF16: return run_tma<TK_BF16, OZ_EPI_STORE>(b, st);
    default: return RHOSVD_ERR_INVALID_ARG;
    }
}

}  // namespace rh

extern "C" int rhosvd_selftest_bits(const double* x, const float* f, const int* e, float* rh, float* rl, double* fd,
                                    float* p2, int n, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !f || !e || !rh || !rl || !fd || !p2))) return RHOSVD_ERR_INVALID_ARG;
    if (n == 0) return RHOSVD_OK;
    const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    rh::k_selftest_bits<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, f, e, rh, rl, fd, p2, n);
    return cudaGetLastError() == cudaSuccess ? RHOSVD_OK : RHOSVD_ERR_CUDA;
}

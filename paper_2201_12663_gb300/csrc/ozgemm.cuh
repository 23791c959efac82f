// ozgemm.cuh -- FP64-class GEMM on the tcgen05 tensor cores by exact digit slicing (used by the
// mixed-precision form of the RHOSVD path).
//
// A real value x with |x| < 2^E is written as x = 2^(E - W) sum_{s=1..S} d_s 2^(-W(s-1)), the d_s
// base-2^W digits of |x| 2^(WS - E) (the last one rounded) carrying the sign of x.  Every digit is
// exact in BF16, every product of two digits exact in FP32 (below 2^(2W)), and a sum of such
// products stays exact while it fits 24 bits.  The product of two operands is
// x y = 2^(Ea + Eb - 2W) sum_{s,t} d_s d'_t 2^(-W(s + t - 2)); the kernels form the groups
// g = s + t up to GMAX in TMEM accumulators and read them back into double-float registers before
// an exact group's FP32 sum could round.  Each operand row gets its own exponent E (from its
// largest entry), so the leading digit carries the row's leading bits.
//   FP64-class products: S = 7 digits of W = 7 bits, GMAX = 9, every group in its own accumulator,
//     exact over its block of 128 K.  The error is the digits' rounding (|x - x^| <= 2^(E - 50))
//     and the dropped pairs s + t >= 10: about 2^-48 of the scaled sum 2^(Ea + Eb) K.
//   Khatri-Rao core: S = 4 digits of W = 8 bits, GMAX = 5, the groups 2 and 3 exact, the groups
//     4 and 5 together in one FP32 accumulator: about 2^-31.
#pragma once
#include "internal.cuh"
#include <cuda_bf16.h>

namespace rh {

constexpr int OZ_BM = 128;      // rows of a CTA tile (TMEM lanes)
constexpr int OZ_BK = 32;       // K granule of a split-K range
constexpr int OZ_NT6 = 64;      // column width that the split-count heuristics count tiles in

// Operand given as digit planes in global memory (bf16 bit patterns), in one of two layouts:
//   row-major (tiles_k == 0): plane p, operand row i, k at base[p * pstride + i * ld + k], ld a
//     multiple of 8;
//   tile-major (tiles_k == KT > 0): rows in tiles of tile_h (128 for an operand on the TMEM lanes,
//     32 for one stacked along N), k in tiles of 16; tile (rt, kt) holds the S planes of its
//     tile_h x 16 block back to back, each in the 32-byte swizzled K-major order the MMA reads
//     (oz_tiled_index), so one stage of an operand is one contiguous copy.
struct OzPlanes {
    const uint16_t* base;
    long long pstride;
    int ld;
    const signed char* exps;   // per operand row exponent E_i (nullable = all `exp0`)
    int exp0;
    int tiles_k;               // tile-major with this many k tiles per row tile (0: row-major)
    int tile_h;                // rows per tile of the tile-major layout (128 or 32)
};

// element (row r, k, plane s) of a tile-major S-plane operand with KT k tiles and H rows per row
// tile: inside an H x 16 plane tile, row r holds 32 bytes whose two 16-byte halves are swapped on
// the rows with bit 2 set (the 32-byte swizzle, anchored to 256-byte boundaries)
__host__ __device__ __forceinline__ long long oz_tiled_index(int S, int KT, int H, int s, int r, int k)
{
    const int rr = r % H, kk = k & 15;
    return ((long long)((r / H) * KT + (k >> 4)) * S + s) * (H * 16) + rr * 16 + (((kk >> 3) ^ ((rr >> 2) & 1)) << 3) +
           (kk & 7);
}

// Generated Khatri-Rao operand for the core: row (j + r2 m), k = nu: V2(j, nu) V3(m, nu)
// (|.| <= 1), each factor given as an FP32 pair (h, l) at V2p[nu ldp + j], V3p[nu ldp + m]
// (consecutive rows j adjacent, so the lanes of a warp, on consecutive rows, read together).
struct OzKR {
    const float2* V2p;
    const float2* V3p;
    int ldp;
    // per-row exponents (|V2(j, .)| < 2^e2[j], |V3(m, .)| < 2^e3[m]): row (j, m) of the operand
    // is cut with E = e2[j] + e3[m], so small rows keep their own 32 bits (null: E = 0)
    const signed char* e2;
    const signed char* e3;
};

struct OzProblem {
    OzPlanes A, B;
    OzKR kr;
    int M, N, K;                 // host values / upper bounds
    const int* dM;
    const int* dN;
    const int* dK;
    int N_from_r2r3;             // core: N = dNa * dNb... (rows of the generated A are r2 r3)
    const int* dNa;
    const int* dNb;
    int M_from_r2r3;             // core: M = r2 * r3 from dNa, dNb
    int krs_from_dNa;            // r2 for the KR row decomposition taken from *dNa
    // output (EPI_STORE): C(i, j) at C[i * crs + j * ccs]; ccs < 0 means ccs = M, crs < 0 means
    // crs = N (sizes decided on the device)
    double* C;
    long long crs, ccs;
    // residual energy (EPI_RESID): sum over the tile of (ref(j, i) - C(i, j))^2, ref element
    // (row j of the reference = operand column j, column i) at ref[i * ref_rs + j * ref_cs]
    const double* ref;
    long long ref_rs, ref_cs;
    double* rpart;
    uint64_t seed;               // Rademacher B: element (k, j) = sign(seed, mode, k, j)
    int mode;
    // split-K (EPI_STORE only): with OzBatch::nsplit > 1, split s sums K range s of nsplit
    // (multiples of 32) into Cpart + s * split_stride, laid out like C; k_oz_reduce then adds
    // the partials into C in a fixed order
    double* Cpart;
    long long split_stride;
    // nullable: the split count decided on the device (sizes known only there), at most
    // OzBatch::nsplit; CTAs of the splits beyond it exit, and 1 writes C directly
    const int* dsplit;
};

struct OzBatch {
    OzProblem p[3];
    int nbatch;
    int nsplit;                  // 0 or 1: no split
    int* err;                    // status word: RHOSVD_ERR_TIMEOUT if a bounded wait gave up
};

enum OzEpi { OZ_EPI_STORE = 0, OZ_EPI_RESID = 1 };

// FP64-class operands are cut into OZ_S64 digits of OZ_W64 bits (49 bits in all); the
// Khatri-Rao core keeps 8-bit digits.  A product of two W-bit digits is below 2^(2W): with W = 7 a
// group of up to 7 digit pairs stays exact in FP32 over 128 K (np 2^14 128 < 2^24).
constexpr int OZ_S64 = 7, OZ_W64 = 7;

// FP32 helpers built from the bits (integer work, no FP64 instruction: GB300 issues those at about
// two lanes a cycle per SM).
// 2^e as a float (subnormal from 2^-149, zero below it, infinity above 2^127)
__device__ __forceinline__ float pow2f(int e)
{
    return e >= -126 ? __int_as_float(min(e + 127, 255) << 23) : (e >= -149 ? __int_as_float(1 << (e + 149)) : 0.f);
}

// x = rh + rl as two floats without FP64 work: rh is x truncated to 24 significant bits, rl the
// rest (up to 29 bits) rounded to a float: |rh + rl - x| <= 2^-48 |x| for |x| >= 2^-97, below
// that the rest leaves FP32's range (an absolute error under 2^-120).  A value outside FP32's
// normal range (|x| < 2^-126; |x| >= 2^128 does not occur, the operands are normalised) gives
// 0 + 0.
__device__ __forceinline__ void split_f64(double x, float& rh, float& rl)
{
    const uint32_t h = (uint32_t)__double2hiint(x), l = (uint32_t)__double2loint(x);
    const uint32_t sgn = h & 0x80000000u;
    const int E = (int)((h >> 20) & 0x7ffu) - 1023;
    const bool ok = E >= -126 && E <= 127;
    const uint32_t fh = sgn | ((uint32_t)(E + 127) << 23) | ((h & 0xfffffu) << 3) | (l >> 29);
    const uint32_t r29 = l & 0x1fffffffu;
    // the 29-bit rest as a float: its two parts are exact (2^23 + d less 2^23), one rounding in the fma
    const float ra = __fsub_rn(__uint_as_float(0x4B000000u | (r29 >> 6)), 8388608.0f);
    const float rb = __fsub_rn(__uint_as_float(0x4B000000u | (r29 & 63u)), 8388608.0f);
    const float rm = __fmul_rn(__fmaf_rn(ra, 64.0f, rb), pow2f(E - 52));
    rh = ok ? __uint_as_float(fh) : 0.f;
    rl = ok ? __uint_as_float(__float_as_uint(rm) | sgn) : 0.f;
}

// S digit planes (bf16 bit patterns) of the signed integer F = +-round(|x| 2^(W S - E)).
// Digit s (s = 1..S) is d 2^(-W(s-1)) with d < 2^W (s > 1) or d <= 2^W (s = 1): at most eight
// significant bits and a power-of-two scale, so the float d * 2^(-W(s-1)) is exact and its bf16
// pattern is the float's upper half (no rounding); the sign is the top bit.
__device__ __forceinline__ void oz_digits_int(long long F, int S, uint16_t* out, int W = 8)
{
    const bool neg = F < 0;
    const unsigned long long A = (unsigned long long)(neg ? -F : F);
    const unsigned sgn = neg ? 0x8000u : 0u;
    for (int s = 1; s <= S; ++s) {
        const unsigned long long mask = s == 1 ? ((2ull << W) - 1) : ((1ull << W) - 1);
        const int d = (int)((A >> (W * (S - s))) & mask);
        // d < 2^23 as a float without a conversion instruction: the float 2^23 + d, less 2^23
        const float fd = __fsub_rn(__int_as_float(0x4B000000 | d), 8388608.0f);
        const float v = fd * __int_as_float((127 - W * (s - 1)) << 23);
        out[s - 1] = d ? (uint16_t)((__float_as_uint(v) >> 16) | sgn) : (uint16_t)0;
    }
}

// digit planes of one FP64 value for exponent E (|x| < 2^E): writes S bf16 bit patterns of
// W-bit digits
__device__ __forceinline__ void oz_digits(double x, int E, int S, uint16_t* out, int W = 8)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7FF);
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    int e;
    if (ef == 0) { e = -1022; } else { m |= 0x10000000000000ull; e = ef - 1023; }
    // |x| = m 2^(e-52); F = round(|x| 2^(W S - E)) = round(m 2^(e - 52 + W S - E))
    const int sh = 52 - (e + W * S - E);
    unsigned long long F;
    if (m == 0 || sh >= 64) {
        F = 0;
    } else if (sh <= 0) {
        F = 1ull << (W * S);     // |x| >= 2^E does not occur for a valid exponent; saturate
    } else {
        F = (m + (1ull << (sh - 1))) >> sh;
    }
    const long long Fs = (long long)F;
    oz_digits_int((bits >> 63) ? -Fs : Fs, S, out, W);
}

// The Khatri-Rao core's digits of one FP64 value for exponent E (|x| < 2^E): the signed integer
// F = +-round(|x| 2^(32 - E)) cut into 4 balanced base-256 digits (each the rounded quotient of the
// remainder, so |d1| <= 256 and |d2|, |d3|, |d4| <= 128), plane s holding d_s 2^(-8(s-1)).  The
// smaller digits keep the core's exact groups exact over 256 K instead of 128 K.
__device__ __forceinline__ void oz_digits_bal(double x, int E, uint16_t* out)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ef = (int)((bits >> 52) & 0x7FF);
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    int e;
    if (ef == 0) { e = -1022; } else { m |= 0x10000000000000ull; e = ef - 1023; }
    const int sh = 52 - (e + 32 - E);
    unsigned long long F;
    if (m == 0 || sh >= 64) F = 0;
    else if (sh <= 0) F = 1ull << 32;          // |x| >= 2^E does not occur for a valid exponent
    else F = (m + (1ull << (sh - 1))) >> sh;
    long long t = (bits >> 63) ? -(long long)F : (long long)F;
#pragma unroll
    for (int s = 1; s <= 4; ++s) {
        const int b = 8 * (4 - s);
        // round half up: floor((t + 2^(b-1)) / 2^b) (an arithmetic shift), the last digit the rest
        const long long d = s < 4 ? (t + (1LL << (b - 1))) >> b : t;
        t -= d << b;
        const int di = (int)d, ad = di < 0 ? -di : di;      // |d| <= 256
        const float v = __fsub_rn(__int_as_float(0x4B000000 | ad), 8388608.0f) * __int_as_float((127 - 8 * (s - 1)) << 23);
        out[s - 1] = (uint16_t)((__float_as_uint(v) >> 16) | (di < 0 ? 0x8000u : 0u));
    }
}

// Digit planes of an operand: operand row i < rows, k < K reads X[i * rs + k * cs] (times
// kscale[k] if given); planes[p * pstride + i * ld + k], zero for k in [K, ld).  With `exps`,
// a per-row exponent E_i (|x| < 2^E_i) is computed and stored, else every row uses exp0.
// One problem per mode b < nb with its own pointers (arrays of 3).
struct OzSliceArgs {
    const double* X[3];
    long long rs[3], cs[3];
    int rows[3];                 // host upper bound
    const int* drows[3];         // nullable device row count
    int K[3];
    const int* dK[3];
    const double* kscale[3];
    uint16_t* planes[3];
    long long pstride[3];
    int ld[3];
    signed char* exps[3];
    int S;
    int exp0;
    // tile-major output (tiles_k[b] > 0): tile_h[b] rows a tile, every k < 16 tiles_k written
    // (zeros past K); optionally a second copy in another layout (planes2[b], tile_h2[b]: a
    // product whose two operands are the same matrix needs it on the lanes and stacked)
    int tiles_k[3];
    int tile_h[3];
    uint16_t* planes2[3];
    int tile_h2[3];
};
int launch_oz_slice(const OzSliceArgs& a, int nb, cudaStream_t st);

// the instantiations: FP64-class product (S = 7 digits of 7 bits, all groups exact) storing C or reducing
// the residual energy; range sketch against Rademacher signs; Khatri-Rao core (S = 4)
enum OzKind { OZ_F64_STORE = 0, OZ_F64_RESID = 1, OZ_SKETCH = 2, OZ_CORE = 3, OZ_BF16 = 4, OZ_SKETCH5 = 5 };
// OZ_SKETCH5: the range sketch with OZ_S_SKETCH5 digits of U~ (35 bits) instead of seven, for the
// tolerances at which its digit error stays far below eps (the choice and its bound: api.cu).
constexpr int OZ_S_SKETCH5 = 5;
// OZ_BF16: one plane per operand holding arbitrary BF16 values (not digits), exponents 8 and 8
// (scale 2^0), FP32 accumulation read back every 256 K: a plain BF16 GEMM with FP64 output,
// used by the learned-proposal network.
int launch_ozgemm(const OzBatch& b, OzKind kind, cudaStream_t st);

// The TMA-fed, warp-specialised form (ozgemm_tma.cu) of the plane-operand kinds OZ_F64_STORE,
// OZ_F64_RESID, OZ_SKETCH and OZ_BF16: whether every operand of the batch can be described by a
// tensor map (16-byte aligned planes, ld a multiple of 8, planes a whole number of rows apart),
// the GEMM launch itself (launch_ozgemm adds the split-K reduction), and its status word.
bool ozgemm_tma_supports(const OzBatch& b, OzKind kind);
int launch_ozgemm_tma(const OzBatch& b, OzKind kind, cudaStream_t st);
int oztma_take_status(cudaStream_t st, int* out);
// tiles (residual partials) of one problem's grid in that form
long long ozgemm_tma_tiles(OzKind kind, int M, int N);
// The Khatri-Rao core (OZ_CORE) in the same form: B (diag(xi') V1 digit planes, S = 4) tile-major
// with 160-row tiles, A generated from OzProblem::kr in the kernel.
constexpr int OZ_CORE_NT = 160;
bool ozcore_tma_supports(const OzBatch& b);
int launch_ozcore_tma(const OzBatch& b, cudaStream_t st);

// status of the products launched with OzBatch::err == nullptr: copies the library's status word
// to *out (RHOSVD_ERR_TIMEOUT after an expired wait, else 0) and clears it; synchronises `st`
int oz_take_status(cudaStream_t st, int* out);

// split count for an M x N x K product: enough CTAs for two per SM, at least 4 stages each
int oz_choose_split(int M, int N, int K, int nt, int nbatch);
// the Khatri-Rao core's split count from the device ranks r (see k_core_split)
int launch_core_split(const int* r, int K, int smax, long long split_stride, int* out, cudaStream_t st);

}  // namespace rh

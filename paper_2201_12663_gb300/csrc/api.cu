// api.cu -- C ABI of the RHOSVD library: argument checks, workspace plan and the stream-
// ordered launch sequence of the canonical-to-Tucker transform (Def. 2.2, Prop. 2.2).
// Every rank decision is taken on the device; the host never synchronises inside a call.
#include "internal.cuh"
#include "ozgemm.cuh"
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <stdio.h>
#include <string.h>

using namespace rh;

// ---------------------------------------------------------------- tracing
// Optional per-stage timing with CUDA events recorded on the call's stream (off by default),
// and a count of kernel launches made by the library.
namespace {
std::atomic<long long> g_launches{0};
std::mutex g_prof_mu;
int g_prof_on = 0;
constexpr int PROF_MAX = 4096;
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
ProfRec g_prof[PROF_MAX];
int g_prof_n = 0;
cudaEvent_t g_pool[2 * PROF_MAX];
int g_pool_n = 0, g_pool_used = 0;
struct ProfAcc {
    const char* name;
    double ms;
    long long count;
};
ProfAcc g_acc[64];
int g_acc_n = 0;

cudaEvent_t pool_event()
{
    if (g_pool_used < g_pool_n) return g_pool[g_pool_used++];
    if (g_pool_n >= 2 * PROF_MAX) return nullptr;
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool[g_pool_n++] = e;
    g_pool_used = g_pool_n;
    return e;
}

char g_prof_filter[64] = {0};
int g_prof_keep = 0;

// an event record that also works while the stream is being captured into a graph (there it
// becomes a record node that every replay executes)
void prof_record(cudaEvent_t e, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

int prof_begin(const char* name, cudaStream_t st)
{
    if (!g_prof_on) return -1;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_filter[0] && strcmp(name, g_prof_filter) != 0) return -1;
    if (g_prof_n >= PROF_MAX) return -1;
    cudaEvent_t a = pool_event(), b = pool_event();
    if (!a || !b) return -1;
    g_prof[g_prof_n] = ProfRec{name, a, b};
    prof_record(a, st);
    return g_prof_n++;
}

void prof_end(int id, cudaStream_t st)
{
    if (id >= 0) prof_record(g_prof[id].b, st);
}
}  // namespace

void rh::count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// An auxiliary stream of a caller's stream, with the two events of a fork and a join: work that
// does not depend on the chain in progress runs on it beside that chain.  Created once per
// (device, caller stream), never while the caller's stream is being captured (then the work stays
// on the caller's stream); at most 64 of them.
struct AuxStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
std::mutex g_aux_mu;
std::map<std::pair<int, cudaStream_t>, AuxStream> g_aux;

bool aux_stream(cudaStream_t st, AuxStream* out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lk(g_aux_mu);
    auto it = g_aux.find({dev, st});
    if (it != g_aux.end()) {
        *out = it->second;
        return true;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone || g_aux.size() >= 64)
        return false;
    AuxStream a;
    if (cudaStreamCreateWithFlags(&a.s, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&a.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&a.join, cudaEventDisableTiming) != cudaSuccess)
        return false;
    g_aux[{dev, st}] = a;
    *out = a;
    return true;
}

#define STAGE(name, call)                     \
    do {                                      \
        const int pid_ = prof_begin(name, st); \
        rc = (call);                          \
        prof_end(pid_, st);                   \
        if (rc) return rc;                    \
    } while (0)

extern "C" long long rhosvd_launch_count(void) { return g_launches.load(); }

extern "C" int rhosvd_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    const int prev = g_prof_on;
    g_prof_on = on ? 1 : 0;
    return prev;
}

// ---- replayable sequences of library calls (CUDA graphs)
namespace {
struct GraphRec {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    long long launches;
};
thread_local long long g_capture_start = -1;
}  // namespace

extern "C" int rhosvd_graph_begin(void* stream)
{
    if (!stream || g_capture_start >= 0) return RHOSVD_ERR_INVALID_ARG;
    if (cudaStreamBeginCapture((cudaStream_t)stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    g_capture_start = g_launches.load();
    return RHOSVD_OK;
}

extern "C" int rhosvd_graph_end(void* stream, void** graph)
{
    if (!stream || !graph || g_capture_start < 0) return RHOSVD_ERR_INVALID_ARG;
    const long long n = g_launches.load() - g_capture_start;
    g_capture_start = -1;
    *graph = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture((cudaStream_t)stream, &g) != cudaSuccess || !g) return RHOSVD_ERR_CUDA;
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return RHOSVD_ERR_CUDA;
    }
    GraphRec* r = new (std::nothrow) GraphRec{g, ex, n};
    if (!r) {
        cudaGraphExecDestroy(ex);
        cudaGraphDestroy(g);
        return RHOSVD_ERR_CUDA;
    }
    g_launches.fetch_sub(n);          // counted again at every replay
    *graph = r;
    return RHOSVD_OK;
}

extern "C" int rhosvd_graph_launch(void* graph, void* stream)
{
    if (!graph) return RHOSVD_ERR_INVALID_ARG;
    GraphRec* r = (GraphRec*)graph;
    if (cudaGraphLaunch(r->exec, (cudaStream_t)stream) != cudaSuccess) return RHOSVD_ERR_CUDA;
    g_launches.fetch_add(r->launches);
    return RHOSVD_OK;
}

extern "C" int rhosvd_graph_destroy(void* graph)
{
    if (!graph) return RHOSVD_OK;
    GraphRec* r = (GraphRec*)graph;
    cudaGraphExecDestroy(r->exec);
    cudaGraphDestroy(r->graph);
    delete r;
    return RHOSVD_OK;
}

extern "C" int rhosvd_profile_keep(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    const int prev = g_prof_keep;
    g_prof_keep = on ? 1 : 0;
    if (!on) {
        g_prof_n = 0;
        g_pool_used = 0;
    }
    return prev;
}

extern "C" int rhosvd_profile_filter(const char* stage)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_filter[0] = 0;
    if (stage) {
        strncpy(g_prof_filter, stage, sizeof(g_prof_filter) - 1);
        g_prof_filter[sizeof(g_prof_filter) - 1] = 0;
    }
    return RHOSVD_OK;
}

extern "C" int rhosvd_profile_read(char* buf, int len)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int i = 0; i < g_prof_n; ++i) {
        if (cudaEventSynchronize(g_prof[i].b) != cudaSuccess) return RHOSVD_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g_prof[i].a, g_prof[i].b) != cudaSuccess) return RHOSVD_ERR_CUDA;
        int j = 0;
        while (j < g_acc_n && strcmp(g_acc[j].name, g_prof[i].name) != 0) ++j;
        if (j == g_acc_n && g_acc_n < 64) g_acc[g_acc_n++] = ProfAcc{g_prof[i].name, 0.0, 0};
        if (j < 64) { g_acc[j].ms += ms; g_acc[j].count += 1; }
    }
    if (!g_prof_keep) {
        g_prof_n = 0;
        g_pool_used = 0;
    }
    int w = 0;
    for (int j = 0; j < g_acc_n && buf && w < len; ++j)
        w += snprintf(buf + w, (size_t)(len - w), "%s %lld %.6f\n", g_acc[j].name, g_acc[j].count, g_acc[j].ms);
    g_acc_n = 0;
    return w;
}

namespace {

constexpr size_t ALIGN = 256;

inline size_t up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Workspace plan: sizes and byte offsets, a pure function of sizes and options.
struct Plan {
    int n[3], R, rmax, kin[3], direct[3];
    int kb[3];            // basis capacity of mode l: k_l, plus kdef for a sketched mode
    int KW;               // basis capacity: max k_l over modes + kdef
    int kdef;             // width of the deflation sketch (0: none)
    int start;            // a caller's start basis replaces the random sketch
    int NQ;               // max n_l over modes
    int ks_sketch, ks_gram, ks_bbt;
    size_t o_cpart, o_colmax, o_defl, o_defT, o_ydf2, o_dpart;
    size_t o_state, o_norms, o_keep, o_nn2, o_Un, o_xin, o_bufA, o_bufB, o_G, o_L, o_perm, o_B, o_vec, o_W, o_V, o_Z, o_rp,
        o_part;
    // mixed-precision form: digit planes and helpers
    int mixed;
    int ldR, ldn, ldk;            // plane row lengths (multiples of 8) for K = R, n, k
    int tkR;                      // k tiles of the tile-major U~ planes with K = R (even)
    int sk5;                      // the range sketches take five digits of U~ (OZ_SKETCH5)
    int tkC;                      // k tiles of the core's diag(xi') V1 planes
    long long sSg;                // per-mode size of the sketch's sign plane (elements)
    size_t o_sgn;
    size_t o_pU1, o_pU2, o_pP1, o_pP2, o_eU2, o_eP1, o_eP2, o_Vt;
    long long EX;         // per-mode stride of the per-row exponent arrays
    int oz_s_sketch, oz_s_gram, oz_s_bbt, oz_s_defl;   // split-K counts of the tensor-core products
    size_t o_ozpart;      // their partial sums
    long long ozpart_n;   // its capacity in doubles
    long long sU1, sU2, sP1, sP2; // per-mode plane-set sizes (elements)
    long long rp_stride;   // residual partials per mode (tiles of the residual GEMM)
    // ALS refinement (als > 0 sweeps): C_l (KW x rmax^2), split-K partials of G_l, energies
    int als, ks_als;
    size_t o_als_C, o_als_part, o_als_e, o_als_q, o_als_k;
    // FP32 outputs: Z and beta are formed in FP64 here, then rounded into the caller's buffers
    int out_fp32;
    size_t o_zf, o_bf;
    size_t total;
};

int choose_split(int tiles, int K)
{
    int ks = (2 * 148 + tiles - 1) / (tiles > 0 ? tiles : 1);
    int kmax = (K + 255) / 256;
    if (ks > kmax) ks = kmax;
    if (ks > 32) ks = 32;
    if (ks < 1) ks = 1;
    return ks;
}

int tiles_of(int M, int N) { return ((M + 63) / 64) * ((N + 63) / 64); }

int make_plan(const rhosvd_cp* cp, const rhosvd_opts* o, Plan* p, int k0 = 0, int als = 0)
{
    if (!cp || !o) return RHOSVD_ERR_INVALID_ARG;
    if (cp->R < 0) return RHOSVD_ERR_INVALID_ARG;
    if (o->r_max < 1 || o->r_max > KMAX || o->oversample < 0) return RHOSVD_ERR_INVALID_ARG;
    if (k0 < 0 || k0 > KMAX - 64) return RHOSVD_ERR_INVALID_ARG;
    if (o->precision != RHOSVD_PLAIN_FP64 && o->precision != RHOSVD_MIXED) return RHOSVD_ERR_INVALID_ARG;
    if (!(o->eps >= 0.0)) return RHOSVD_ERR_INVALID_ARG;
    if (o->out_fp32 != 0 && o->out_fp32 != 1) return RHOSVD_ERR_INVALID_ARG;
    memset(p, 0, sizeof(*p));
    p->R = cp->R;
    p->rmax = o->r_max;
    int kcap = o->r_max + o->oversample;
    if (kcap > KMAX) kcap = KMAX;
    // width of the deflation sketch; the basis may grow to kin + kdef columns
    int kdef = o->deflate == 0 ? 16 : (o->deflate < 0 ? 0 : o->deflate);
    if (kdef > 64) return RHOSVD_ERR_INVALID_ARG;
    if (kcap + kdef > KMAX) kdef = KMAX - kcap;
    p->KW = 1;
    p->NQ = 1;
    for (int l = 0; l < 3; ++l) {
        if (cp->n[l] < 1 || cp->ld[l] < cp->n[l] || o->ranks[l] < 0) return RHOSVD_ERR_INVALID_ARG;
        p->n[l] = cp->n[l];
        if (cp->n[l] <= kcap) {
            p->direct[l] = 1;
            p->kin[l] = cp->n[l];
        } else {
            p->direct[l] = 0;
            int k = k0 > 0 ? k0 : kcap;             // a start basis fixes the subspace width
            if (cp->R > 0 && k > cp->R) k = cp->R;
            if (k < 1) k = 1;
            p->kin[l] = k;
        }
        if (p->kin[l] > p->KW) p->KW = p->kin[l];
        if (cp->n[l] > p->NQ) p->NQ = cp->n[l];
    }
    p->kdef = 0;
    for (int l = 0; l < 3; ++l)
        if (!p->direct[l] && cp->R > p->kin[l]) p->kdef = kdef;   // only a sketched mode can miss directions
    if (p->kdef > 0 && p->KW + p->kdef > KMAX) p->kdef = KMAX - p->KW;
    p->start = k0 > 0;
    for (int l = 0; l < 3; ++l) p->kb[l] = p->kin[l] + (p->direct[l] ? 0 : p->kdef);
    p->KW += p->kdef;
    const int R = cp->R > 0 ? cp->R : 1;
    const long long NK = (long long)p->NQ * p->KW, KK = (long long)p->KW * p->KW;
    // split-K factors of the launches that use the partial buffer
    int t_sk = 0, t_g = 0;
    for (int l = 0; l < 3; ++l) {
        t_sk += tiles_of(p->n[l], p->kin[l]);
        t_g += tiles_of(p->kin[l], p->kin[l]);
    }
    p->ks_sketch = choose_split(t_sk, R);
    p->ks_gram = choose_split(t_g, p->NQ);
    p->ks_bbt = choose_split(t_g, R);
    long long part = 0;
    part = (long long)p->ks_sketch * 3 * NK;
    long long pg = (long long)p->ks_gram * 3 * KK, pb = (long long)p->ks_bbt * 3 * KK;
    if (pg > part) part = pg;
    if (pb > part) part = pb;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o2 = off; off += up(bytes); return o2; };
    p->o_state = take(sizeof(DevState));
    p->o_norms = take(sizeof(double) * 3 * R);
    p->o_colmax = take(sizeof(double) * 3 * R);
    p->o_keep = take(sizeof(double) * R);
    p->o_nn2 = take(sizeof(double) * 3 * R);
    p->o_Un = take(sizeof(double) * 3 * (size_t)p->NQ * R);
    p->o_xin = take(sizeof(double) * R);
    p->o_bufA = take(sizeof(double) * 3 * NK);
    p->o_bufB = take(sizeof(double) * 3 * NK);
    p->o_G = take(sizeof(double) * 3 * KK);
    p->o_L = take(sizeof(double) * 3 * KK);
    p->o_perm = take(sizeof(int) * 3 * p->KW);
    p->o_B = take(sizeof(double) * 3 * (size_t)p->KW * R);
    p->o_vec = take(sizeof(double) * 6 * 3 * p->KW);
    p->o_W = take(sizeof(double) * 3 * KK);
    p->o_V = take(sizeof(double) * 3 * (size_t)p->KW * R);
    p->o_Z = take(sizeof(double) * 3 * NK);
    p->rp_stride = (long long)((p->NQ + 63) / 64) * ((R + 63) / 64);
    if (o->precision == RHOSVD_MIXED) {
        const long long t = rh::ozgemm_tma_tiles(rh::OZ_F64_RESID, p->NQ, R);
        if (t > p->rp_stride) p->rp_stride = t;
    }
    p->o_rp = take(sizeof(double) * 3 * (size_t)p->rp_stride);
    p->o_cpart = take(sizeof(double) * 3 * (size_t)rh::RITZ_CHUNKS * rh::KMAX);
    if (p->kdef > 0) {
        p->o_defl = take(sizeof(double) * 3 * (size_t)NK);
        p->o_defT = take(sizeof(double) * 3 * (size_t)rh::KMAX * p->kdef);
        // the deflation sketch's own output, so that it can run beside the first CholeskyQR
        if (o->precision == RHOSVD_MIXED) p->o_ydf2 = take(sizeof(double) * 3 * (size_t)NK);
    }
    p->o_part = take(sizeof(double) * (size_t)part);
    p->mixed = (o->precision == RHOSVD_MIXED);
    if (p->mixed) {
        auto up8 = [](long long x) { return (int)((x + 7) / 8 * 8); };
        p->ldR = up8(R);
        p->ldn = up8(p->NQ);
        p->ldk = up8(p->KW);
        // the two digit-plane sets of U~ are tile-major (whole 128 x 16 tiles, see ozgemm.cuh):
        // U1 rows x, k = nu; U2 rows nu, k = x
        p->tkR = (R + 31) / 32 * 2;     // an even count: the sketch streams k tiles in pairs
        // Five digits of U~ for the range sketch where their error cannot matter at the
        // requested eps: the sketch of U~ + E with |E_ij| <= 2^-35 (fixed exponent 1, 35 bits)
        // finds a basis whose projection error exceeds U~'s own by at most ||E||_F <= 2^-35
        // sqrt(n) ||U~||_F (unit columns), and the residual energy that decides the ranks is
        // measured on U~ itself afterwards.  With eps >= 1.5e-9 sqrt(n) that is at most 2% of
        // eps ||U~||_F, 4e-4 of the threshold energy: a rank moves only at a tie that close.
        // Every rank chosen by eps; otherwise, and below that eps, seven digits.
        bool by_eps = true;
        for (int l = 0; l < 3; ++l) by_eps = by_eps && o->ranks[l] == 0;
        p->sk5 = by_eps && o->eps >= 1.5e-9 * sqrt((double)p->NQ);
        p->sU1 = (long long)OZ_S64 * ((p->NQ + 127) / 128 * 128) * (p->tkR * 16LL);
        p->sU2 = (long long)OZ_S64 * ((R + 127) / 128 * 128) * ((p->NQ + 15) / 16 * 16LL);
        // the small operands' plane sets (tile-major: rows padded to 128, k to 16; enough for
        // the row-major layout too)
        auto tsz = [](long long rows, long long K) { return (rows + 127) / 128 * 128 * ((K + 15) / 16 * 16); };
        long long pm = tsz(R, p->KW);
        const long long cand[4] = {tsz(p->KW, R), tsz(p->KW, p->KW), tsz(p->KW, p->NQ), tsz(p->NQ, p->KW)};
        for (long long c : cand) pm = c > pm ? c : pm;
        p->sP1 = (long long)OZ_S64 * pm;
        p->sP2 = (long long)OZ_S64 * pm;
        // the core's diag(xi') V1 planes: 4 planes, 160-row tiles, k tiles of 16
        p->tkC = (R + 15) / 16;
        const long long rc = p->rmax < p->KW ? p->rmax : p->KW;
        const long long score = 4LL * ((rc + OZ_CORE_NT - 1) / OZ_CORE_NT * OZ_CORE_NT) * (p->tkC * 16LL);
        if (score > p->sP2) p->sP2 = score;
        p->o_pU1 = take(sizeof(uint16_t) * 3 * (size_t)p->sU1);
        p->o_pU2 = take(sizeof(uint16_t) * 3 * (size_t)p->sU2);
        p->o_pP1 = take(sizeof(uint16_t) * 3 * (size_t)p->sP1);
        p->o_pP2 = take(sizeof(uint16_t) * 3 * (size_t)p->sP2);
        long long ex = p->NQ > R ? p->NQ : R;
        p->EX = ex > p->KW ? ex : p->KW;
        p->o_eU2 = take(3 * (size_t)p->EX);
        p->o_eP1 = take(3 * (size_t)p->EX);
        p->o_eP2 = take(3 * (size_t)p->EX);
        p->o_Vt = take(sizeof(double) * 3 * (size_t)R * p->KW);
        // the sketch's signs as tile-major BF16 planes (rows = sketch columns)
        p->sSg = (long long)((p->KW + 127) / 128 * 128) * (p->tkR * 16LL);
        p->o_sgn = take(sizeof(uint16_t) * 3 * (size_t)p->sSg);
        int nsk = 0;
        for (int l = 0; l < 3; ++l) nsk += p->direct[l] ? 0 : 1;
        p->oz_s_sketch = nsk > 0 ? rh::oz_choose_split((int)p->NQ, p->KW, R, 96, nsk) : 1;
        p->oz_s_gram = nsk > 0 ? rh::oz_choose_split(p->KW, p->KW, (int)p->NQ, rh::OZ_NT6, nsk) : 1;
        // the deflation sketch's split partials have a buffer of their own (it may run beside the
        // chain, whose products use the common one): n x kdef a mode and split
        p->oz_s_defl = (nsk > 0 && p->kdef > 0) ? rh::oz_choose_split((int)p->NQ, p->kdef, R, 96, nsk) : 1;
        if (p->kdef > 0 && p->oz_s_defl > 1)
            p->o_dpart = take(sizeof(double) * 3 * (size_t)p->oz_s_defl * (size_t)p->NQ * p->kdef);
        p->oz_s_bbt = rh::oz_choose_split(p->KW, p->KW, R, rh::OZ_NT6, 3);
        long long zp = 3LL * p->oz_s_sketch * NK;
        if (3LL * p->oz_s_gram * KK > zp) zp = 3LL * p->oz_s_gram * KK;
        if (3LL * p->oz_s_bbt * KK > zp) zp = 3LL * p->oz_s_bbt * KK;
        p->o_ozpart = take(sizeof(double) * (size_t)zp);
        p->ozpart_n = zp;
    }
    p->als = als;
    if (als > 0) {
        const long long KC = (long long)p->rmax * p->rmax;
        p->ks_als = choose_split(tiles_of(p->KW, p->KW), (int)KC);
        p->o_als_C = take(sizeof(double) * (size_t)p->KW * (size_t)KC);
        p->o_als_part = take(sizeof(double) * (size_t)p->ks_als * KK);
        p->o_als_e = take(sizeof(double) * 6 * (size_t)als);
        p->o_als_q = take(sizeof(double) * rh::KMAX);
        p->o_als_k = take(sizeof(int) * 3);
    }
    p->out_fp32 = o->out_fp32;
    if (p->out_fp32) {
        p->o_zf = take(sizeof(double) * 3 * (size_t)p->NQ * p->rmax);
        p->o_bf = take(sizeof(double) * (size_t)p->rmax * p->rmax * p->rmax);
    }
    p->total = off;
    return RHOSVD_OK;
}

GemmProblem blank_problem()
{
    GemmProblem g;
    memset(&g, 0, sizeof(g));
    return g;
}

// Tile-major digit planes for the TMA-fed products: problem b of a slice call writes tiles of H
// rows (LANE: the operand on the TMEM lanes; COL: the one stacked along N), and the operand handed
// to the product describes the same layout.
constexpr int LANE = rh::OZ_BM, COL = 32;

void tiled_out(OzSliceArgs& s, int b, int H)
{
    s.tiles_k[b] = (s.K[b] + 15) / 16;
    s.tile_h[b] = H;
}

OzPlanes planes_of(const OzSliceArgs& s, int b)
{
    return OzPlanes{s.planes[b], s.pstride[b], s.ld[b], s.exps[b], s.exp0, s.tiles_k[b], s.tile_h[b]};
}

// the second copy of a dual-layout slice
OzPlanes planes2_of(const OzSliceArgs& s, int b)
{
    return OzPlanes{s.planes2[b], s.pstride[b], s.ld[b], s.exps[b], s.exp0, s.tiles_k[b], s.tile_h2[b]};
}

}  // namespace

extern "C" int rhosvd_version(void) { return 100; }

extern "C" const char* rhosvd_strerror(int code)
{
    switch (code) {
    case RHOSVD_OK: return "success";
    case RHOSVD_ERR_INVALID_ARG: return "invalid argument";
    case RHOSVD_ERR_RANK_OVERFLOW: return "a Tucker rank exceeds r_max (needed rank in info->r_needed)";
    case RHOSVD_ERR_NOT_CONVERGED: return "a small factorisation broke down";
    case RHOSVD_ERR_NONFINITE: return "non-finite value in the factors or weights";
    case RHOSVD_ERR_SKETCH: return "the range sketch missed more energy than eps allows (raise oversample or r_max)";
    case RHOSVD_ERR_CUDA: return "CUDA runtime or launch error";
    case RHOSVD_ERR_WORKSPACE: return "workspace missing or too small";
    case RHOSVD_ERR_TIMEOUT: return "a bounded wait inside a kernel gave up";
    case RHOSVD_ERR_SCRATCH_LIMIT:
        return "problem needs more scratch than the static buffer of rhosvd_c2t_noalloc holds (use rhosvd_c2t)";
    default: return "unknown status";
    }
}

extern "C" size_t rhosvd_c2t_workspace_size(const rhosvd_cp* cp, const rhosvd_opts* opts)
{
    Plan p;
    if (make_plan(cp, opts, &p) != RHOSVD_OK) return 0;
    return p.total;
}

extern "C" int rhosvd_subspace_width(const rhosvd_cp* cp, const rhosvd_opts* opts, int mode)
{
    Plan p;
    if (mode < 0 || mode > 2 || make_plan(cp, opts, &p) != RHOSVD_OK) return -1;
    return p.kin[mode];
}

struct StartBasis {
    const double* Q0[3];   // n_l x k0, column-major, leading dimension ld[l]
    int ld[3];
    int k0;
    int iters;             // 0: Y = Q0; 1: Y = U~ (U~^T Q0)
};

// Second factor of a Hadamard product reduced without storing it: cp holds the first factor's
// columns with R = Ra Rb, and term nu = i + Ra j is cp's column i times b's column j.
struct HadSrc {
    const rhosvd_cp* b;
    int Ra;
    const double* xa;
};

namespace {

// One reduction in flight: the call's arguments, its plan, the workspace's named regions and the
// stream.  Each stage of the path is one member function; run() calls them in the path's order,
// and the first error ends the call.
struct Reduction {
    const rhosvd_cp* cp = nullptr;
    const rhosvd_opts* opts = nullptr;
    const StartBasis* sb0 = nullptr;
    const rhosvd_tucker* out = nullptr;
    const HadSrc* had = nullptr;
    Plan p;
    cudaStream_t st = nullptr;
    char* ws = nullptr;
    int rc = 0;
    // workspace regions and sizes (bind)
    DevState* S = nullptr;
    double *norms, *colmax, *keepf, *nn2, *Un, *xin, *bufA, *bufB, *G, *L;
    int* perm;
    double *Bm, *vec, *W, *Vw, *Zw, *rpart, *part;
    int R = 0, KW = 0, rmax = 0;
    long long NK = 0, KK = 0;
    int vs = 0;
    double *vd, *ve, *vtau, *vD, *vL, *vmu;
    long long VS = 0, US = 0;
    bool mixed = false;
    uint16_t *pU1, *pU2, *pP1, *pP2;
    signed char *eU2, *eP1, *eP2;
    long long EX = 0;
    double* Vt;
    uint16_t* sgn;
    double* ozpart;
    int* ozerr;
    // Z and beta as formed here: the caller's buffers, or FP64 staging for FP32 outputs (reset)
    double* Zout[3];
    double* beta_out = nullptr;
    // the modes (all three, the sketched ones) and the basis each mode ends with (direct_bases)
    ModeMap all, sk;
    int nsk = 0;
    double* Qfin[3];
    int ldq[3];

    void bind(void* workspace, void* stream);
    int reset();
    int normalise();
    int direct_bases();
    int slice_sketch_operand();
    int sketch();
    int cholqr3(double* bIn, double* bTmp, const int* kh, const int* dk0, int* dm, int* dkx, double* d0out,
                const double* d0ref, double floor_rel, int* dnear, const AuxStream* fork_to = nullptr,
                double* fork_ydf = nullptr);
    int deflation_sketch(cudaStream_t st, double* Ydf);
    int range_basis();
    int project();
    int eigen();
    int bases_residual();
    int rank_final();
    int als();
    int outputs_core();
    int to_fp32();
    int run();
};

// the workspace's named regions and the sizes every stage uses
void Reduction::bind(void* workspace, void* stream)
{
    st = (cudaStream_t)stream;
    ws = (char*)workspace;
    S = (DevState*)(ws + p.o_state);
    norms = (double*)(ws + p.o_norms);
    colmax = (double*)(ws + p.o_colmax);
    keepf = (double*)(ws + p.o_keep);
    nn2 = (double*)(ws + p.o_nn2);
    Un = (double*)(ws + p.o_Un);
    xin = (double*)(ws + p.o_xin);
    bufA = (double*)(ws + p.o_bufA);
    bufB = (double*)(ws + p.o_bufB);
    G = (double*)(ws + p.o_G);
    L = (double*)(ws + p.o_L);
    perm = (int*)(ws + p.o_perm);
    Bm = (double*)(ws + p.o_B);
    vec = (double*)(ws + p.o_vec);
    W = (double*)(ws + p.o_W);
    Vw = (double*)(ws + p.o_V);
    Zw = (double*)(ws + p.o_Z);
    rpart = (double*)(ws + p.o_rp);
    part = (double*)(ws + p.o_part);
    R = cp->R;
    KW = p.KW;
    rmax = p.rmax;
    NK = (long long)p.NQ * KW;
    KK = (long long)KW * KW;
    vs = KW;
    vd = vec;
    ve = vec + 3 * vs;
    vtau = vec + 6 * vs;
    vD = vec + 9 * vs;
    vL = vec + 12 * vs;
    vmu = vec + 15 * vs;
    VS = (long long)KW * (R > 0 ? R : 1);
    US = (long long)p.NQ * (R > 0 ? R : 1);   // normalised side matrix per mode
    mixed = p.mixed != 0;
    pU1 = mixed ? (uint16_t*)(ws + p.o_pU1) : nullptr;     // U planes, rows x, k = nu
    pU2 = mixed ? (uint16_t*)(ws + p.o_pU2) : nullptr;     // U planes, rows nu, k = x
    pP1 = mixed ? (uint16_t*)(ws + p.o_pP1) : nullptr;
    pP2 = mixed ? (uint16_t*)(ws + p.o_pP2) : nullptr;
    // per-row exponents of the digit planes (one array per plane buffer, stride EX per mode)
    eU2 = mixed ? (signed char*)(ws + p.o_eU2) : nullptr;
    eP1 = mixed ? (signed char*)(ws + p.o_eP1) : nullptr;
    eP2 = mixed ? (signed char*)(ws + p.o_eP2) : nullptr;
    EX = mixed ? p.EX : 0;
    Vt = mixed ? (double*)(ws + p.o_Vt) : nullptr;
    sgn = mixed ? (uint16_t*)(ws + p.o_sgn) : nullptr;
    ozpart = mixed ? (double*)(ws + p.o_ozpart) : nullptr;
    ozerr = &out->info->status;
}

// outputs and device state cleared; the state counters set
int Reduction::reset()
{
    // ---- reset outputs and state
    if (cudaMemsetAsync(out->info, 0, sizeof(rhosvd_info), st) != cudaSuccess) return RHOSVD_ERR_CUDA;
    if (cudaMemsetAsync(S, 0, sizeof(DevState), st) != cudaSuccess) return RHOSVD_ERR_CUDA;
    // Z and beta as formed here: the caller's buffers, or FP64 staging for FP32 outputs
    beta_out = p.out_fp32 ? (double*)(ws + p.o_bf) : (double*)out->beta;
    for (int l = 0; l < 3; ++l) {
        Zout[l] = p.out_fp32 ? (double*)(ws + p.o_zf) + (size_t)l * p.NQ * rmax : (double*)out->Z[l];
        if (cudaMemsetAsync(Zout[l], 0, sizeof(double) * (size_t)p.n[l] * rmax, st) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
        if (cudaMemsetAsync(out->sigma[l], 0, sizeof(double) * KMAX, st) != cudaSuccess) return RHOSVD_ERR_CUDA;
    }
    STAGE("init_state", launch_init_state(S, p.kin[0], p.kin[1], p.kin[2], p.direct[0] ? p.n[0] : 0,
                                p.direct[1] ? p.n[1] : 0, p.direct[2] ? p.n[2] : 0, p.kdef, st));
    return RHOSVD_OK;
}

// a1: column norms, dropped terms, normalised weights and side matrices
int Reduction::normalise()
{
    // ---- a1: column norms, normalised weights (Sec. 2.1)
    NormArgs na;
    memset(&na, 0, sizeof(na));
    for (int l = 0; l < 3; ++l) { na.U[l] = cp->U[l]; na.ld[l] = cp->ld[l]; na.n[l] = p.n[l]; }
    na.R = R;
    if (had) {
        for (int l = 0; l < 3; ++l) { na.B[l] = had->b->U[l]; na.ldb[l] = had->b->ld[l]; }
        na.Ra = had->Ra;
        na.xa = had->xa;
        na.xb = had->b->xi;
    }
    na.norms = norms;
    na.colmax = colmax;
    STAGE("colnorms", launch_colnorms(na, st));
    // the mixed form cuts the projection operand's digit planes (rows nu, k = x, per-row
    // exponents) while it writes the normalised columns
    NormSlice ns;
    memset(&ns, 0, sizeof(ns));
    if (mixed) {
        for (int l = 0; l < 3; ++l) {
            ns.planes[l] = pU2 + l * p.sU2;
            ns.pstride[l] = (long long)R * p.ldn;
            ns.ld[l] = p.ldn;
            ns.exps[l] = eU2 + l * EX;
            ns.tiles_k[l] = (p.n[l] + 15) / 16;
            ns.tile_h[l] = LANE;                   // on the TMEM lanes of the projection
        }
    }
    STAGE("normalize", launch_terms(na, cp->xi, keepf, xin, out->xi_out, out->info, Un, US, nn2, S->total, ns, st));
    return RHOSVD_OK;
}

// the modes that are sketched, and the identity basis of the direct ones
int Reduction::direct_bases()
{
    all = ModeMap{{0, 1, 2}};
    nsk = 0;
    for (int l = 0; l < 3; ++l)
        if (!p.direct[l]) sk.m[nsk++] = l;
    for (int l = 0; l < 3; ++l) {
        ldq[l] = p.n[l];
        if (p.direct[l]) {
            Qfin[l] = bufA + l * NK;
            STAGE("identity", launch_identity(Qfin[l], p.n[l], p.n[l], st));
        } else {
            Qfin[l] = bufB + l * NK;
        }
    }
    return RHOSVD_OK;
}

// the range sketch's operand as digit planes (mixed form)
int Reduction::slice_sketch_operand()
{
    if (mixed && R > 0 && nsk > 0) {
        // digit planes of the range-sketch operand (rows x, k = nu): one fixed exponent (the
        // normalised entries are below 2^1), which is all a random range sketch needs
        SliceTArgs sb;
        memset(&sb, 0, sizeof(sb));
        sb.E0 = 1;
        sb.S = p.sk5 ? OZ_S_SKETCH5 : OZ_S64;
        int nmax = 0;
        for (int b = 0; b < nsk; ++b) {
            const int l = sk.m[b];
            sb.X[b] = Un + l * US;
            sb.ldx[b] = p.n[l];
            sb.rows[b] = p.n[l];
            sb.K[b] = R;
            sb.planes[b] = pU1 + l * p.sU1;
            sb.pstride[b] = (long long)p.n[l] * p.ldR;
            sb.ld[b] = p.tkR * 16;                 // every k of the last tile written (zeros past R)
            sb.tiles_k[b] = p.tkR;
            sb.tile_h[b] = COL;                    // stacked along N in the sketches
            nmax = p.n[l] > nmax ? p.n[l] : nmax;
        }
        STAGE("slice_u", launch_slice_t(sb, nsk, p.tkR * 16, nmax, st));
    }
    return RHOSVD_OK;
}

// a2: range sketch Y = U~ Omega (Rademacher) into bufA, or the caller's start basis
int Reduction::sketch()
{
    if (nsk > 0 && R > 0) {
        // ---- a2: range sketch Y = U diag(1/||u||) Omega (Rademacher), Y in bufA
        GemmBatch gb;
        memset(&gb, 0, sizeof(gb));
        gb.nbatch = nsk;
        gb.ksplit = p.ks_sketch;
        gb.bkind = B_SKETCH;
        for (int b = 0; b < nsk; ++b) {
            const int l = sk.m[b];
            GemmProblem g = blank_problem();
            g.A = Mat{Un + l * US, 1, (long long)p.n[l]};
            g.C = bufA + l * NK;
            g.crs = 1;
            g.ccs = p.n[l];
            g.M = p.n[l];
            g.N = p.kin[l];
            g.K = R;
            g.seed = opts->seed;
            g.mode = l;
            gb.p[b] = g;
        }
        if (p.start && sb0->iters == 0) {
            // the caller's start basis itself is orthonormalised (no pass over U~)
            for (int b = 0; b < nsk; ++b) {
                const int l = sk.m[b];
                if (cudaMemcpy2DAsync(bufA + l * NK, sizeof(double) * p.n[l], sb0->Q0[l], sizeof(double) * sb0->ld[l],
                                      sizeof(double) * p.n[l], p.kin[l], cudaMemcpyDeviceToDevice, st) != cudaSuccess)
                    return RHOSVD_ERR_CUDA;
            }
        } else if (p.start) {
            // one subspace iteration from the caller's start basis replaces the random sketch:
            // P = U~^T Q0 (R x k0, column-major in the B buffer), Y = U~ P
            if (mixed) {
                OzSliceArgs sq, sp;
                memset(&sq, 0, sizeof(sq));
                memset(&sp, 0, sizeof(sp));
                sq.S = sp.S = OZ_S64;
                OzBatch o1, o2;
                memset(&o1, 0, sizeof(o1));
                memset(&o2, 0, sizeof(o2));
                o1.nbatch = o2.nbatch = nsk;
                o1.err = o2.err = ozerr;
                for (int b = 0; b < nsk; ++b) {
                    const int l = sk.m[b];
                    double* P = Bm + (size_t)l * KW * R;
                    sq.X[b] = sb0->Q0[l];
                    sq.rs[b] = sb0->ld[l];
                    sq.cs[b] = 1;
                    sq.rows[b] = p.kin[l];
                    sq.K[b] = p.n[l];
                    sq.planes[b] = pP2 + l * p.sP2;
                    sq.pstride[b] = (long long)p.kin[l] * p.ldn;
                    sq.ld[b] = p.ldn;
                    sq.exps[b] = eP2 + l * EX;
                    tiled_out(sq, b, COL);
                    OzProblem& q = o1.p[b];
                    q.A = OzPlanes{pU2 + l * p.sU2, (long long)R * p.ldn, p.ldn, eU2 + l * EX, 0, (p.n[l] + 15) / 16, LANE};
                    q.B = planes_of(sq, b);
                    q.M = R;
                    q.N = p.kin[l];
                    q.K = p.n[l];
                    q.C = P;
                    q.crs = 1;
                    q.ccs = R;
                    sp.X[b] = P;
                    sp.rs[b] = R;
                    sp.cs[b] = 1;
                    sp.rows[b] = p.kin[l];
                    sp.K[b] = R;
                    sp.planes[b] = pP1 + l * p.sP1;
                    sp.pstride[b] = (long long)p.kin[l] * p.ldR;
                    sp.ld[b] = p.ldR;
                    sp.exps[b] = eP1 + l * EX;
                    // Y^T = P^T U~^T: the rows j of P on the TMEM lanes, the tile-major planes
                    // of U~ (rows x) stacked, Y(x, j) stored at x + n j
                    tiled_out(sp, b, LANE);
                    OzProblem& q2 = o2.p[b];
                    q2.A = planes_of(sp, b);
                    q2.B = OzPlanes{pU1 + l * p.sU1, (long long)p.n[l] * p.ldR, p.ldR, nullptr, 1, p.tkR, COL};
                    q2.M = p.kin[l];
                    q2.N = p.n[l];
                    q2.K = R;
                    q2.C = bufA + l * NK;
                    q2.crs = p.n[l];
                    q2.ccs = 1;
                }
                STAGE("sketch", launch_oz_slice(sq, nsk, st));
                STAGE("sketch", launch_ozgemm(o1, OZ_F64_STORE, st));
                STAGE("sketch", launch_oz_slice(sp, nsk, st));
                STAGE("sketch", launch_ozgemm(o2, OZ_F64_STORE, st));
            } else {
                GemmBatch g1, g2;
                memset(&g1, 0, sizeof(g1));
                g1.nbatch = nsk;
                g1.ksplit = 1;
                g1.bkind = B_PLAIN;
                g2 = g1;
                for (int b = 0; b < nsk; ++b) {
                    const int l = sk.m[b];
                    double* P = Bm + (size_t)l * KW * R;
                    GemmProblem a = blank_problem();
                    a.A = Mat{Un + l * US, (long long)p.n[l], 1};            // A(nu, x) = U~(x, nu)
                    a.B = Mat{sb0->Q0[l], 1, (long long)sb0->ld[l]};       // B(x, j) = Q0(x, j)
                    a.C = P;
                    a.crs = 1;
                    a.ccs = R;
                    a.M = R;
                    a.N = p.kin[l];
                    a.K = p.n[l];
                    g1.p[b] = a;
                    GemmProblem c = blank_problem();
                    c.A = Mat{Un + l * US, 1, (long long)p.n[l]};            // A(x, nu) = U~(x, nu)
                    c.B = Mat{P, 1, (long long)R};                          // B(nu, j) = P(nu, j)
                    c.C = bufA + l * NK;
                    c.crs = 1;
                    c.ccs = p.n[l];
                    c.M = p.n[l];
                    c.N = p.kin[l];
                    c.K = R;
                    g2.p[b] = c;
                }
                STAGE("sketch", launch_gemm(g1, st));
                STAGE("sketch", launch_gemm(g2, st));
            }
        } else if (mixed) {
            OzBatch ob;
            memset(&ob, 0, sizeof(ob));
            ob.nbatch = nsk;
            ob.nsplit = p.oz_s_sketch;
            ob.err = ozerr;
            SignPlaneArgs sg;
            memset(&sg, 0, sizeof(sg));
            sg.tiles_k = p.tkR;
            sg.seed = opts->seed;
            int kmx = 0;
            for (int b = 0; b < nsk; ++b) {
                const int l = sk.m[b];
                sg.planes[b] = sgn + l * p.sSg;
                sg.rows[b] = p.kin[l];
                sg.K[b] = R;
                sg.mode[b] = l;
                kmx = p.kin[l] > kmx ? p.kin[l] : kmx;
            }
            STAGE("sketch", launch_sign_planes(sg, nsk, kmx, st));
            for (int b = 0; b < nsk; ++b) {
                const int l = sk.m[b];
                OzProblem& q = ob.p[b];
                q.B = OzPlanes{sgn + l * p.sSg, 0, 0, nullptr, 0, p.tkR, LANE};
                q.A = OzPlanes{pU1 + l * p.sU1, (long long)p.n[l] * p.ldR, p.ldR, nullptr, 1, p.tkR, COL};
                q.M = p.n[l];
                q.N = p.kin[l];
                q.K = R;
                q.C = bufA + l * NK;
                q.crs = 1;
                q.ccs = p.n[l];
                q.seed = opts->seed;
                q.mode = l;
                q.Cpart = ozpart + (size_t)l * p.oz_s_sketch * NK;
                q.split_stride = NK;
            }
            STAGE("sketch", launch_ozgemm(ob, p.sk5 ? OZ_SKETCH5 : OZ_SKETCH, st));
        } else {
            STAGE("sketch", launch_gemm_splitk(gb, part, st));
        }
    }
    return RHOSVD_OK;
}

// a3: CholeskyQR with pivoting, three passes: bIn -> bTmp -> bIn -> bTmp.  kh: host
// column bounds; dk0: device columns of the input; dm, dkx: device basis width and input
// columns (outputs); d0out: the first pass's largest Gram diagonal (optional); d0ref,
// floor_rel: absolute pivot floor floor_rel * d0ref (optional); fork_to: the deflation sketch into
// fork_ydf is launched on that auxiliary stream right after the first pass's Cholesky, once the
// Cholesky's clusters hold their SMs (optional)
int Reduction::cholqr3(double* bIn, double* bTmp, const int* kh, const int* dk0, int* dm, int* dkx, double* d0out,
                       const double* d0ref, double floor_rel, int* dnear, const AuxStream* fork_to, double* fork_ydf)
{
    const double tols[3] = {1e-15, 1e-11, 0.0};
    const int pivots[3] = {1, 1, 0};
    for (int pass = 0; pass < 3; ++pass) {
        double* X = (pass == 1) ? bTmp : bIn;
        double* Y = (pass == 1) ? bIn : bTmp;
        GemmBatch g2;
        memset(&g2, 0, sizeof(g2));
        g2.nbatch = nsk;
        g2.ksplit = p.ks_gram;
        g2.bkind = B_PLAIN;
        for (int b = 0; b < nsk; ++b) {
            const int l = sk.m[b];
            GemmProblem g = blank_problem();
            double* Xl = X + l * NK;
            g.A = Mat{Xl, (long long)p.n[l], 1};      // A(i,x) = X(x,i)
            g.B = Mat{Xl, 1, (long long)p.n[l]};      // B(x,j) = X(x,j)
            g.C = G + l * KK;
            g.crs = 1;
            g.ccs = KW;
            g.M = kh[l];
            g.N = kh[l];
            g.K = p.n[l];
            if (pass > 0) { g.dM = &dm[l]; g.dN = &dm[l]; }
            g2.p[b] = g;
        }
        if (mixed) {
            // G = X^T X on the tensor cores: rows c of the operand = columns of X (k = x);
            // every digit group is exact, so the Gram keeps FP64-class accuracy
            OzSliceArgs sg;
            memset(&sg, 0, sizeof(sg));
            sg.S = OZ_S64;
            OzBatch ob;
            memset(&ob, 0, sizeof(ob));
            ob.nbatch = nsk;
            ob.nsplit = p.oz_s_gram;
            ob.err = ozerr;
            for (int b = 0; b < nsk; ++b) {
                const int l = sk.m[b];
                sg.X[b] = X + l * NK;
                sg.rs[b] = p.n[l];
                sg.cs[b] = 1;
                sg.rows[b] = kh[l];
                sg.drows[b] = pass > 0 ? &dm[l] : nullptr;
                sg.K[b] = p.n[l];
                sg.planes[b] = pP2 + l * p.sP2;
                sg.pstride[b] = (long long)kh[l] * p.ldn;
                sg.ld[b] = p.ldn;
                sg.exps[b] = eP2 + l * EX;
                tiled_out(sg, b, LANE);
                sg.planes2[b] = pP1 + l * p.sP1;     // the same planes stacked along N
                sg.tile_h2[b] = COL;
                OzProblem& q = ob.p[b];
                q.A = planes_of(sg, b);
                q.B = planes2_of(sg, b);
                q.M = q.N = kh[l];
                if (pass > 0) q.dM = q.dN = &dm[l];
                q.K = p.n[l];
                q.C = G + l * KK;
                q.crs = 1;
                q.ccs = KW;
                q.Cpart = ozpart + (size_t)l * p.oz_s_gram * KK;
                q.split_stride = KK;
            }
            STAGE("cholqr_gram", launch_oz_slice(sg, nsk, st));
            STAGE("cholqr_gram", launch_ozgemm(ob, OZ_F64_STORE, st));
        } else {
            STAGE("cholqr_gram", launch_gemm_splitk(g2, part, st));
        }
        const int* dk = (pass == 0) ? dk0 : dm;
        // Y = X P Lt^{-T}: the triangular inverse scattered into W (the Gram's buffer), then
        // one GEMM over the kx columns of X (a near-identity Gram has W written by the Cholesky)
        double* Wq = G;
        STAGE("cholqr_chol", launch_chol(sk, G, KK, KW, dk, dkx, L, KK, KW, perm, KW, dm, S->piv_fail,
                                         pivots[pass], tols[pass], nsk, KW, pass == 0 ? d0out : nullptr,
                                         d0ref, floor_rel, Wq, KK, KW, dnear, st));
        if (pass == 0 && fork_to) {
            if (cudaEventRecord(fork_to->fork, st) != cudaSuccess ||
                cudaStreamWaitEvent(fork_to->s, fork_to->fork, 0) != cudaSuccess)
                return RHOSVD_ERR_CUDA;
            rc = deflation_sketch(fork_to->s, fork_ydf);
            if (rc) return rc;
            if (cudaEventRecord(fork_to->join, fork_to->s) != cudaSuccess) return RHOSVD_ERR_CUDA;
        }
        STAGE("cholqr_trinv", launch_trinv(sk, L, KK, KW, perm, KW, dkx, dm, Wq, KK, KW, dnear, nsk, st));
        if (mixed) {
            OzSliceArgs sx, sw;
            memset(&sx, 0, sizeof(sx));
            memset(&sw, 0, sizeof(sw));
            sx.S = sw.S = OZ_S64;
            OzBatch ob;
            memset(&ob, 0, sizeof(ob));
            ob.nbatch = nsk;
            ob.err = ozerr;
            for (int b = 0; b < nsk; ++b) {
                const int l = sk.m[b];
                sx.X[b] = X + l * NK;                 // rows x, k = column c of X
                sx.rs[b] = 1;
                sx.cs[b] = p.n[l];
                sx.rows[b] = p.n[l];
                sx.K[b] = kh[l];
                sx.dK[b] = &dkx[l];
                sx.planes[b] = pP2 + l * p.sP2;
                sx.pstride[b] = (long long)p.n[l] * p.ldk;
                sx.ld[b] = p.ldk;
                sx.exps[b] = eP2 + l * EX;
                sw.X[b] = Wq + l * KK;                // rows t (columns of W), k = c
                sw.rs[b] = KW;
                sw.cs[b] = 1;
                sw.rows[b] = kh[l];
                sw.drows[b] = &dm[l];
                sw.K[b] = kh[l];
                sw.dK[b] = &dkx[l];
                sw.planes[b] = pP1 + l * p.sP1;
                sw.pstride[b] = (long long)kh[l] * p.ldk;
                sw.ld[b] = p.ldk;
                sw.exps[b] = eP1 + l * EX;
                tiled_out(sx, b, LANE);
                tiled_out(sw, b, COL);
                OzProblem& q = ob.p[b];
                q.A = planes_of(sx, b);
                q.B = planes_of(sw, b);
                q.M = p.n[l];
                q.N = kh[l];
                q.dN = &dm[l];
                q.K = kh[l];
                q.dK = &dkx[l];
                q.C = Y + l * NK;
                q.crs = 1;
                q.ccs = p.n[l];
            }
            STAGE("cholqr_apply", launch_oz_slice(sx, nsk, st));
            STAGE("cholqr_apply", launch_oz_slice(sw, nsk, st));
            STAGE("cholqr_apply", launch_ozgemm(ob, OZ_F64_STORE, st));
        } else {
            GemmBatch gq;
            memset(&gq, 0, sizeof(gq));
            gq.nbatch = nsk;
            gq.ksplit = 1;
            gq.bkind = B_PLAIN;
            for (int b = 0; b < nsk; ++b) {
                const int l = sk.m[b];
                GemmProblem g = blank_problem();
                g.A = Mat{X + l * NK, 1, (long long)p.n[l]};      // A(x, c) = X(x, c)
                g.B = Mat{Wq + l * KK, 1, (long long)KW};         // B(c, t) = W(c, t)
                g.C = Y + l * NK;
                g.crs = 1;
                g.ccs = p.n[l];
                g.M = p.n[l];
                g.N = kh[l];
                g.dN = &dm[l];
                g.K = kh[l];
                g.dK = &dkx[l];
                gq.p[b] = g;
            }
            STAGE("cholqr_apply", launch_gemm(gq, st));
        }
    }
    return 0;
}

// the deflation sketch Y2 = U~ Omega2 into Ydf (projected afterwards), on stream st.  It does not
// depend on the first basis, so the mixed form runs it on an auxiliary stream beside the first
// CholeskyQR; its split partials have a buffer of their own, and its split count is the same
// whether it runs there or not, so that both schedules give the same bits
int Reduction::deflation_sketch(cudaStream_t st, double* Ydf)
{
    const unsigned long long seed2 = opts->seed ^ 0x9E3779B97F4A7C15ull;
    if (mixed) {
        OzBatch ob;
        memset(&ob, 0, sizeof(ob));
        ob.nbatch = nsk;
        ob.nsplit = p.oz_s_defl;
        ob.err = ozerr;
        SignPlaneArgs sg;
        memset(&sg, 0, sizeof(sg));
        sg.tiles_k = p.tkR;
        sg.seed = seed2;
        for (int b = 0; b < nsk; ++b) {
            const int l = sk.m[b];
            sg.planes[b] = sgn + l * p.sSg;
            sg.rows[b] = p.kdef;
            sg.K[b] = R;
            sg.mode[b] = l;
        }
        STAGE("deflate_sketch", launch_sign_planes(sg, nsk, p.kdef, st));
        for (int b = 0; b < nsk; ++b) {
            const int l = sk.m[b];
            OzProblem& q = ob.p[b];
            q.B = OzPlanes{sgn + l * p.sSg, 0, 0, nullptr, 0, p.tkR, LANE};
            q.A = OzPlanes{pU1 + l * p.sU1, (long long)p.n[l] * p.ldR, p.ldR, nullptr, 1, p.tkR, COL};
            q.M = p.n[l];
            q.N = p.kdef;
            q.K = R;
            q.C = Ydf + l * NK;
            q.crs = 1;
            q.ccs = p.n[l];
            q.seed = seed2;
            q.mode = l;
            q.Cpart = p.oz_s_defl > 1 ? (double*)(ws + p.o_dpart) + (size_t)l * p.oz_s_defl * p.NQ * p.kdef : nullptr;
            q.split_stride = (long long)p.NQ * p.kdef;
        }
        STAGE("deflate_sketch", launch_ozgemm(ob, p.sk5 ? OZ_SKETCH5 : OZ_SKETCH, st));
    } else {
        GemmBatch gd;
        memset(&gd, 0, sizeof(gd));
        gd.nbatch = nsk;
        gd.ksplit = p.ks_sketch;
        gd.bkind = B_SKETCH;
        for (int b = 0; b < nsk; ++b) {
            const int l = sk.m[b];
            GemmProblem g = blank_problem();
            g.A = Mat{Un + l * US, 1, (long long)p.n[l]};
            g.C = Ydf + l * NK;
            g.crs = 1;
            g.ccs = p.n[l];
            g.M = p.n[l];
            g.N = p.kdef;
            g.K = R;
            g.seed = seed2;
            g.mode = l;
            gd.p[b] = g;
        }
        STAGE("deflate_sketch", launch_gemm_splitk(gd, part, st));
    }
    return RHOSVD_OK;
}

// a3: the first basis by pivoted CholeskyQR (the deflation sketch beside it), then the deflation
int Reduction::range_basis()
{
    if (nsk > 0 && R > 0) {
        AuxStream aux;
        const bool fork = mixed && p.kdef > 0 && p.o_ydf2 != 0 && aux_stream(st, &aux);
        double* const Ydf = fork ? (double*)(ws + p.o_ydf2) : bufA;   // bufA: free after the first CholeskyQR
        {
            const int rc = cholqr3(bufA, bufB, p.kin, S->kin, S->m, S->kx, S->gmax, nullptr, 0.0, S->near,
                                   fork ? &aux : nullptr, Ydf);
            if (rc) return rc;
        }
        if (p.kdef > 0) {
            // ---- deflation: a second sketch on the residual of the first basis,
            // Y2 = (I - Q Q^T) U Omega2 (two projections), orthonormalised on its own scale and
            // appended to Q.  A Gram of one sketch resolves directions only down to ~sqrt(u) of
            // the largest; near eps = 1e-7 the tail energy sits there.  A pivot must also exceed
            // 1e-26 of the first sketch's largest Gram diagonal: below that, Y2 is rounding noise.
            double* Qdf = (double*)(ws + p.o_defl);
            double* Tdf = (double*)(ws + p.o_defT);
            int kdh[3] = {p.kdef, p.kdef, p.kdef};
            if (fork) {
                if (cudaStreamWaitEvent(st, aux.join, 0) != cudaSuccess) return RHOSVD_ERR_CUDA;
            } else {
                rc = deflation_sketch(st, Ydf);
                if (rc) return rc;
            }
            for (int it = 0; it < 2; ++it)
                STAGE("deflate_project", launch_deflate(sk, bufB, Ydf, NK, p.n, S->m, p.kdef, Tdf,
                                                        (long long)KMAX * p.kdef, nsk, p.NQ, st));
            {
                const int rc = cholqr3(Ydf, Qdf, kdh, S->kdef, S->mdef, S->kxdef, nullptr, S->gmax, 1e-26,
                                       S->neardef);
                if (rc) return rc;
            }
            STAGE("deflate_append", launch_append(sk, bufB, Qdf, NK, p.n, S->m, S->mdef, nsk, p.NQ, p.kdef, st));
        }
    }
    return RHOSVD_OK;
}

// a4, a5: projection B = Q^T U~ and its Gram M = B B^T
int Reduction::project()
{
    if (R > 0) {
        // ---- a4: projection B = Q^T U diag(1/||u||)  (m_l x R, ld KW)
        GemmBatch gb;
        memset(&gb, 0, sizeof(gb));
        gb.nbatch = 3;
        gb.ksplit = 1;
        gb.bkind = B_PLAIN;
        for (int l = 0; l < 3; ++l) {
            GemmProblem g = blank_problem();
            g.A = Mat{Qfin[l], (long long)ldq[l], 1};
            g.B = Mat{Un + l * US, 1, (long long)p.n[l]};
            g.C = Bm + (size_t)l * KW * R;
            g.crs = 1;
            g.ccs = KW;
            g.M = p.kb[l];
            g.dM = &S->m[l];
            g.N = R;
            g.K = p.n[l];
            gb.p[l] = g;
        }
        if (mixed) {
            OzSliceArgs sq;
            memset(&sq, 0, sizeof(sq));
            sq.S = OZ_S64;
            OzBatch ob;
            memset(&ob, 0, sizeof(ob));
            ob.nbatch = 3;
            ob.err = ozerr;
            for (int l = 0; l < 3; ++l) {
                sq.X[l] = Qfin[l];
                sq.rs[l] = ldq[l];
                sq.cs[l] = 1;
                sq.rows[l] = p.kb[l];
                sq.drows[l] = &S->m[l];
                sq.K[l] = p.n[l];
                sq.planes[l] = pP2 + l * p.sP2;
                sq.pstride[l] = (long long)p.kb[l] * p.ldn;
                sq.ld[l] = p.ldn;
                sq.exps[l] = eP2 + l * EX;
                OzProblem& q = ob.p[l];
                tiled_out(sq, l, COL);
                q.A = OzPlanes{pU2 + l * p.sU2, (long long)R * p.ldn, p.ldn, eU2 + l * EX, 0, (p.n[l] + 15) / 16, LANE};
                q.B = planes_of(sq, l);
                q.M = R;
                q.N = p.kb[l];
                q.dN = &S->m[l];
                q.K = p.n[l];
                q.C = Bm + (size_t)l * KW * R;
                q.crs = KW;
                q.ccs = 1;
            }
            STAGE("project_slice", launch_oz_slice(sq, 3, st));
            STAGE("project", launch_ozgemm(ob, OZ_F64_STORE, st));
        } else {
            STAGE("project", launch_gemm(gb, st));
        }

        // ---- a5: M = B B^T (m_l x m_l), trace, tridiagonal form, eigenvalues
        GemmBatch gm;
        memset(&gm, 0, sizeof(gm));
        gm.nbatch = 3;
        gm.ksplit = p.ks_bbt;
        gm.bkind = B_PLAIN;
        for (int l = 0; l < 3; ++l) {
            GemmProblem g = blank_problem();
            double* Bl = Bm + (size_t)l * KW * R;
            g.A = Mat{Bl, 1, KW};
            g.B = Mat{Bl, KW, 1};
            g.C = G + l * KK;
            g.crs = 1;
            g.ccs = KW;
            g.M = p.kb[l];
            g.N = p.kb[l];
            g.K = R;
            g.dM = &S->m[l];
            g.dN = &S->m[l];
            gm.p[l] = g;
        }
        if (mixed) {
            // M = B B^T on the tensor cores: rows i of B (k = nu, stride KW)
            OzSliceArgs sg;
            memset(&sg, 0, sizeof(sg));
            sg.S = OZ_S64;
            OzBatch ob;
            memset(&ob, 0, sizeof(ob));
            ob.nbatch = 3;
            ob.nsplit = p.oz_s_bbt;
            ob.err = ozerr;
            for (int l = 0; l < 3; ++l) {
                sg.X[l] = Bm + (size_t)l * KW * R;
                sg.rs[l] = 1;
                sg.cs[l] = KW;
                sg.rows[l] = p.kb[l];
                sg.drows[l] = &S->m[l];
                sg.K[l] = R;
                sg.planes[l] = pP1 + l * p.sP1;
                sg.pstride[l] = (long long)p.kb[l] * p.ldR;
                sg.ld[l] = p.ldR;
                sg.exps[l] = eP1 + l * EX;
                tiled_out(sg, l, LANE);
                sg.planes2[l] = pP2 + l * p.sP2;       // the same planes stacked along N
                sg.tile_h2[l] = COL;
                OzProblem& q = ob.p[l];
                q.A = planes_of(sg, l);
                q.B = planes2_of(sg, l);
                q.M = q.N = p.kb[l];
                q.dM = q.dN = &S->m[l];
                q.K = R;
                q.C = G + l * KK;
                q.crs = 1;
                q.ccs = KW;
                q.Cpart = ozpart + (size_t)l * p.oz_s_bbt * KK;
                q.split_stride = KK;
            }
            STAGE("gram_bbt", launch_oz_slice(sg, 3, st));
            STAGE("gram_bbt", launch_ozgemm(ob, OZ_F64_STORE, st));
        } else {
            STAGE("gram_bbt", launch_gemm_splitk(gm, part, st));
        }
    }
    return RHOSVD_OK;
}

// a5, a6: tridiagonal eigen-solver, provisional rank, eigenvectors
int Reduction::eigen()
{
    if (R == 0 && cudaMemsetAsync(G, 0, sizeof(double) * 3 * KK, st) != cudaSuccess) return RHOSVD_ERR_CUDA;
    STAGE("trace", launch_trace(all, G, KK, KW, S->m, S->trace, 3, st));
    STAGE("tridiag", launch_tridiag(all, G, KK, KW, S->m, vd, ve, vtau, vs, 3, KW, st));
    STAGE("eigvals", launch_eigvals(all, vd, ve, vs, S->m, vD, vL, vmu, S, 3, st));

    // ---- a6: provisional rank from the eigenvalues, then eigenvectors of the rhi leading
    //          eigenvalues (rank candidates 0..rhi) and their Householder back-transformation
    RankArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.mu = vmu;
    ra.vstride = vs;
    ra.dk = S->m;
    ra.trace = S->trace;
    ra.total = S->total;
    ra.eps = opts->eps;
    ra.r_max = rmax;
    ra.info = out->info;
    ra.st = S;
    ra.kept = &out->info->kept;
    ra.margin = 16;
    for (int l = 0; l < 3; ++l) {
        ra.ranks[l] = opts->ranks[l];
        ra.sigma[l] = out->sigma[l];
        ra.direct[l] = p.direct[l];
    }
    STAGE("rank_provisional", launch_rank(ra, st));
    STAGE("eigvecs", launch_eigvecs(all, vD, vL, vmu, vs, S->m, S, W, KK, KW, KW, 3, st));
    STAGE("backtransform", launch_backtransform(all, G, KK, KW, vtau, vs, S->m, S, W, KK, KW, KW, 3, st));
    return RHOSVD_OK;
}

// Z_hi = Q W, V_hi = W^T B and the residual energy of every rank candidate
int Reduction::bases_residual()
{
    if (R > 0) {
        // ---- Z_hi = Q W (n_l x rhi, ld n_l) and V_hi = W^T B (rhi x R, ld KW)
        GemmBatch gz;
        memset(&gz, 0, sizeof(gz));
        gz.nbatch = 3;
        gz.ksplit = 1;
        gz.bkind = B_PLAIN;
        GemmBatch gv = gz, gr = gz;
        for (int l = 0; l < 3; ++l) {
            double* Wl = W + l * KK;
            GemmProblem g = blank_problem();
            g.A = Mat{Qfin[l], 1, (long long)ldq[l]};
            g.B = Mat{Wl, 1, KW};
            g.C = Zw + l * NK;
            g.crs = 1;
            g.ccs = p.n[l];
            g.M = p.n[l];
            g.N = p.kb[l];
            g.dN = &S->rhi[l];
            g.K = p.kb[l];
            g.dK = &S->m[l];
            gz.p[l] = g;
            GemmProblem h = blank_problem();
            h.A = Mat{Wl, KW, 1};
            h.B = Mat{Bm + (size_t)l * KW * R, 1, KW};
            h.C = Vw + l * VS;
            h.crs = 1;
            h.ccs = KW;
            h.M = p.kb[l];
            h.dM = &S->rhi[l];
            h.N = R;
            h.K = p.kb[l];
            h.dK = &S->m[l];
            gv.p[l] = h;
            // residual energy ||U_normalised - Z_hi V_hi||_F^2 (no output matrix)
            GemmProblem e = blank_problem();
            e.A = Mat{Zw + l * NK, 1, (long long)p.n[l]};
            e.B = Mat{Vw + l * VS, 1, KW};
            e.M = p.n[l];
            e.N = R;
            e.K = p.kb[l];
            e.dK = &S->rhi[l];
            e.rref = Un + l * US;
            e.rref_ld = p.n[l];
            e.rpart = rpart + l * p.rp_stride;
            gr.p[l] = e;
        }
        if (mixed) {
            // Z_hi = Q W on the tensor cores: rows x of Q (k = i), rows j of W^T (k = i)
            OzSliceArgs sq, sw;
            memset(&sq, 0, sizeof(sq));
            memset(&sw, 0, sizeof(sw));
            sq.S = sw.S = OZ_S64;
            OzBatch oz;
            memset(&oz, 0, sizeof(oz));
            oz.nbatch = 3;
            oz.err = ozerr;
            for (int l = 0; l < 3; ++l) {
                sq.X[l] = Qfin[l];
                sq.rs[l] = 1;
                sq.cs[l] = ldq[l];
                sq.rows[l] = p.n[l];
                sq.K[l] = p.kb[l];
                sq.dK[l] = &S->m[l];
                sq.planes[l] = pP2 + l * p.sP2;
                sq.pstride[l] = (long long)p.n[l] * p.ldk;
                sq.ld[l] = p.ldk;
                sq.exps[l] = eP2 + l * EX;
                sw.X[l] = W + l * KK;
                sw.rs[l] = KW;
                sw.cs[l] = 1;
                sw.rows[l] = p.kb[l];
                sw.drows[l] = &S->rhi[l];
                sw.K[l] = p.kb[l];
                sw.dK[l] = &S->m[l];
                sw.planes[l] = pP1 + l * p.sP1;
                sw.pstride[l] = (long long)p.kb[l] * p.ldk;
                sw.ld[l] = p.ldk;
                sw.exps[l] = eP1 + l * EX;
                tiled_out(sq, l, LANE);
                tiled_out(sw, l, COL);
                OzProblem& q = oz.p[l];
                q.A = planes_of(sq, l);
                q.B = planes_of(sw, l);
                q.M = p.n[l];
                q.N = p.kb[l];
                q.dN = &S->rhi[l];
                q.K = p.kb[l];
                q.dK = &S->m[l];
                q.C = Zw + l * NK;
                q.crs = 1;
                q.ccs = p.n[l];
            }
            STAGE("z_hi", launch_oz_slice(sq, 3, st));
            STAGE("z_hi", launch_oz_slice(sw, 3, st));
            STAGE("z_hi", launch_ozgemm(oz, OZ_F64_STORE, st));
        } else {
            STAGE("z_hi", launch_gemm(gz, st));
        }
        if (mixed) {
            // V_hi (rhi x R, ld KW) = W^T B: rows nu of B (k = i) times rows j of W (k = i)
            OzSliceArgs s1, s2;
            memset(&s1, 0, sizeof(s1));
            memset(&s2, 0, sizeof(s2));
            s1.S = s2.S = OZ_S64;
            OzBatch ob;
            memset(&ob, 0, sizeof(ob));
            ob.nbatch = 3;
            ob.err = ozerr;
            for (int l = 0; l < 3; ++l) {
                s1.X[l] = Bm + (size_t)l * KW * R;
                s1.rs[l] = KW;
                s1.cs[l] = 1;
                s1.rows[l] = R;
                s1.K[l] = p.kb[l];
                s1.dK[l] = &S->m[l];
                s1.planes[l] = pP1 + l * p.sP1;
                s1.pstride[l] = (long long)R * p.ldk;
                s1.ld[l] = p.ldk;
                s2.X[l] = W + l * KK;
                s2.rs[l] = KW;
                s2.cs[l] = 1;
                s2.rows[l] = p.kb[l];
                s2.drows[l] = &S->rhi[l];
                s2.K[l] = p.kb[l];
                s2.dK[l] = &S->m[l];
                s2.planes[l] = pP2 + l * p.sP2;
                s2.pstride[l] = (long long)p.kb[l] * p.ldk;
                s2.ld[l] = p.ldk;
                s1.exps[l] = eP1 + l * EX;
                s2.exps[l] = eP2 + l * EX;
                tiled_out(s1, l, LANE);
                tiled_out(s2, l, COL);
                OzProblem& q = ob.p[l];
                q.A = planes_of(s1, l);
                q.B = planes_of(s2, l);
                q.M = R;
                q.N = p.kb[l];
                q.dN = &S->rhi[l];
                q.K = p.kb[l];
                q.dK = &S->m[l];
                q.C = Vw + l * VS;
                q.crs = KW;
                q.ccs = 1;
            }
            STAGE("v_slice", launch_oz_slice(s1, 3, st));
            STAGE("v_slice", launch_oz_slice(s2, 3, st));
            STAGE("v_hi", launch_ozgemm(ob, OZ_F64_STORE, st));
            // residual energy ||U - Z_hi V_hi||^2: rows nu of V_hi (k = j) times rows x of Z_hi
            OzBatch orb;
            memset(&orb, 0, sizeof(orb));
            orb.nbatch = 3;
            orb.err = ozerr;
            for (int l = 0; l < 3; ++l) {
                s1.X[l] = Vw + l * VS;
                s1.rs[l] = KW;
                s1.cs[l] = 1;
                s1.rows[l] = R;
                s1.K[l] = p.kb[l];
                s1.dK[l] = &S->rhi[l];
                s1.planes[l] = pP1 + l * p.sP1;
                s1.pstride[l] = (long long)R * p.ldk;
                s1.ld[l] = p.ldk;
                s2.X[l] = Zw + l * NK;
                s2.rs[l] = 1;
                s2.cs[l] = p.n[l];
                s2.rows[l] = p.n[l];
                s2.drows[l] = nullptr;
                s2.K[l] = p.kb[l];
                s2.dK[l] = &S->rhi[l];
                s2.planes[l] = pP2 + l * p.sP2;
                s2.pstride[l] = (long long)p.n[l] * p.ldk;
                s2.ld[l] = p.ldk;
                s1.exps[l] = eP1 + l * EX;
                s2.exps[l] = eP2 + l * EX;
                // (U~ - Z V)^T: operand rows x (Z) on the TMEM lanes, columns nu (V), so that the
                // epilogue's reads of U~(x, nu) are consecutive across a warp
                tiled_out(s2, l, LANE);
                tiled_out(s1, l, COL);
                OzProblem& q = orb.p[l];
                q.A = planes_of(s2, l);
                q.B = planes_of(s1, l);
                q.M = p.n[l];
                q.N = R;
                q.K = p.kb[l];
                q.dK = &S->rhi[l];
                q.ref = Un + l * US;
                q.ref_rs = 1;
                q.ref_cs = p.n[l];
                q.rpart = rpart + l * p.rp_stride;
            }
            STAGE("resid_slice", launch_oz_slice(s1, 3, st));
            STAGE("resid_slice", launch_oz_slice(s2, 3, st));
            // every partial the final rank sums starts at zero, whatever grid the product runs on
            if (cudaMemsetAsync(rpart, 0, sizeof(double) * 3 * p.rp_stride, st) != cudaSuccess) return RHOSVD_ERR_CUDA;
            STAGE("residual", launch_ozgemm(orb, OZ_F64_RESID, st));
        } else {
            STAGE("v_hi", launch_gemm(gv, st));
            STAGE("residual", launch_gemm(gr, st));
        }
    } else if (cudaMemsetAsync(rpart, 0, sizeof(double) * 3 * p.rp_stride, st) != cudaSuccess) {
        return RHOSVD_ERR_CUDA;
    }
    return RHOSVD_OK;
}

// a6: the final eps-rank from the residual and the Ritz energies
int Reduction::rank_final()
{
    // ---- final eps-rank (Thm. 2.3) from the residual and the Ritz energies
    FinalArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.V = Vw;
    fa.vstride = VS;
    fa.ldv = KW;
    fa.R = R;
    fa.eps = opts->eps;
    fa.r_max = rmax;
    fa.info = out->info;
    fa.st = S;
    fa.rpart = rpart;
    fa.rpstride = p.rp_stride;
    fa.cpart = (double*)(ws + p.o_cpart);
    fa.nchunk = R > 0 ? (R + 63) / 64 : 1;
    if (fa.nchunk > rh::RITZ_CHUNKS) fa.nchunk = rh::RITZ_CHUNKS;
    for (int l = 0; l < 3; ++l) {
        fa.ranks[l] = opts->ranks[l];
        fa.n[l] = p.n[l];
        fa.ntiles[l] = (int)p.rp_stride;
    }
    STAGE("rank_final", launch_rank_final(fa, st));
    return RHOSVD_OK;
}

// optional ALS sweeps inside the bases Q_l
int Reduction::als()
{
    if (R > 0 && p.als > 0) {
        // ---- ALS refinement (eq. can_A_Tuck_als), modes 0, 1, 2 in turn, inside the basis Q_l:
        //      C_l = B_l diag(xi') (V_m2 (.) V_m1)^T, G_l = C_l C_l^T, W_l = its r_l leading
        //      eigenvectors, V_l = W_l^T B_l; at the end Z_l = Q_l W_l.  The ranks stay r_l.
        double* Cb = (double*)(ws + p.o_als_C);
        double* Gpart = (double*)(ws + p.o_als_part);
        double* Eh = (double*)(ws + p.o_als_e);
        double* qpart = (double*)(ws + p.o_als_q);
        int* kk = (int*)(ws + p.o_als_k);
        const int KC = rmax * rmax;
        for (int sw = 0; sw < p.als; ++sw) {
            for (int l = 0; l < 3; ++l) {
                const int m1 = l == 0 ? 1 : 0, m2 = l == 2 ? 1 : 2;
                const int step = 3 * sw + l;
                ModeMap one = {{l, l, l}};
                double* Bl = Bm + (size_t)l * KW * R;
                double* Gl = G + l * KK;
                double* Wl = W + l * KK;
                STAGE("als_prep", launch_als_set(S, l, kk, st));
                GemmBatch gcb;
                memset(&gcb, 0, sizeof(gcb));
                gcb.nbatch = 1;
                gcb.ksplit = 1;
                gcb.bkind = B_KR;
                GemmProblem c = blank_problem();
                c.A = Mat{Bl, 1, KW};
                c.C = Cb;
                c.crs = 1;
                c.ccs = KW;
                c.M = p.kb[l];
                c.dM = &S->m[l];
                c.N = KC;
                c.N_from_r2r3 = 1;
                c.dNa = &S->r[m1];
                c.dNb = &S->r[m2];
                c.K = R;
                c.V2 = Vw + m1 * VS;
                c.V3 = Vw + m2 * VS;
                c.xi = xin;
                c.ldv = KW;
                gcb.p[0] = c;
                STAGE("als_contract", launch_gemm(gcb, st));
                GemmBatch ggb;
                memset(&ggb, 0, sizeof(ggb));
                ggb.nbatch = 1;
                ggb.ksplit = p.ks_als;
                ggb.bkind = B_PLAIN;
                GemmProblem g = blank_problem();
                g.A = Mat{Cb, 1, KW};
                g.B = Mat{Cb, KW, 1};
                g.C = Gl;
                g.crs = 1;
                g.ccs = KW;
                g.M = g.N = p.kb[l];
                g.dM = g.dN = &S->m[l];
                g.K = KC;
                g.dK = &kk[l];
                ggb.p[0] = g;
                STAGE("als_gram", launch_gemm_splitk(ggb, Gpart, st));
                STAGE("als_energy", launch_als_energy_before(Gl, KW, Wl, KW, &S->m[l], &S->r[l], rmax, qpart,
                                                             Eh + 2 * step, st));
                STAGE("als_eig", launch_tridiag(one, G, KK, KW, S->m, vd, ve, vtau, vs, 1, KW, st));
                STAGE("als_eig", launch_eigvals(one, vd, ve, vs, S->m, vD, vL, vmu, S, 1, st));
                STAGE("als_eig", launch_eigvecs(one, vD, vL, vmu, vs, S->m, S, W, KK, KW, KW, 1, st));
                STAGE("als_eig", launch_backtransform(one, G, KK, KW, vtau, vs, S->m, S, W, KK, KW, KW, 1, st));
                STAGE("als_energy", launch_als_energy_after(vmu + l * vs, S, l, Eh + 2 * step + 1, st));
                GemmBatch gvb;
                memset(&gvb, 0, sizeof(gvb));
                gvb.nbatch = 1;
                gvb.ksplit = 1;
                gvb.bkind = B_PLAIN;
                GemmProblem h = blank_problem();
                h.A = Mat{Wl, KW, 1};
                h.B = Mat{Bl, 1, KW};
                h.C = Vw + l * VS;
                h.crs = 1;
                h.ccs = KW;
                h.M = p.kb[l];
                h.dM = &S->r[l];
                h.N = R;
                h.K = p.kb[l];
                h.dK = &S->m[l];
                gvb.p[0] = h;
                STAGE("als_v", launch_gemm(gvb, st));
            }
        }
        GemmBatch gzb;
        memset(&gzb, 0, sizeof(gzb));
        gzb.nbatch = 3;
        gzb.ksplit = 1;
        gzb.bkind = B_PLAIN;
        for (int l = 0; l < 3; ++l) {
            GemmProblem g = blank_problem();
            g.A = Mat{Qfin[l], 1, (long long)ldq[l]};
            g.B = Mat{W + l * KK, 1, KW};
            g.C = Zw + l * NK;
            g.crs = 1;
            g.ccs = p.n[l];
            g.M = p.n[l];
            g.N = p.kb[l];
            g.dN = &S->r[l];
            g.K = p.kb[l];
            g.dK = &S->m[l];
            gzb.p[l] = g;
        }
        STAGE("als_z", launch_gemm(gzb, st));
    }
    return RHOSVD_OK;
}

// outputs Z (and V), a7: the Khatri-Rao core
int Reduction::outputs_core()
{
    if (R > 0) {
        // ---- outputs: Z = Z_hi(:, :r), optional V = V_hi(:r, :)
        double* zd[3] = {Zout[0], Zout[1], Zout[2]};
        int zld[3] = {p.n[0], p.n[1], p.n[2]};
        STAGE("copy_out", launch_copy2d(Zw, NK, zld, zd, zld, nullptr, p.n, S->r, nullptr, st));
        if (out->V[0] && out->V[1] && out->V[2]) {
            double* vd2[3] = {out->V[0], out->V[1], out->V[2]};
            int vld[3] = {rmax, rmax, rmax};
            int RR[3] = {R, R, R};
            int vls[3] = {KW, KW, KW};
            STAGE("copy_out", launch_copy2d(Vw, VS, vls, vd2, vld, S->r, nullptr, nullptr, RR, st));
        }

        // ---- a7: core beta = V1 diag(xi') (V3 (.) V2)^T (Prop. 2.2), packed r1 x r2 x r3
        GemmBatch gc;
        memset(&gc, 0, sizeof(gc));
        gc.nbatch = 1;
        gc.ksplit = 1;
        gc.bkind = B_KR;
        GemmProblem g = blank_problem();
        g.A = Mat{Vw, 1, KW};
        g.C = beta_out;
        g.crs = 1;
        g.ccs = -1;           // = r1, decided on the device
        g.M = rmax;
        g.dM = &S->r[0];
        g.N = rmax * rmax;
        g.N_from_r2r3 = 1;
        g.dNa = &S->r[1];
        g.dNb = &S->r[2];
        g.K = R;
        g.V2 = Vw + VS;
        g.V3 = Vw + 2 * VS;
        g.xi = xin;
        g.ldv = KW;
        gc.p[0] = g;
        if (mixed) {
            // V^(2), V^(3) as FP32 pairs (same layout as V) for the generated Khatri-Rao operand,
            // and the digit planes of diag(xi') V^(1) (rows i, k = nu, per-row exponents)
            const long long VTS = (long long)R * KW;
            STAGE("core_prep", launch_split_v(Vw, VS, KW, (float2*)Vt, VTS, KW, R, S->r, 1, 2, st));
            // per-row exponents of V^(2), V^(3) (modes 1, 2 of eP1): the Khatri-Rao row (j, m)
            // is cut with e2[j] + e3[m]
            STAGE("core_prep", launch_row_exps((const float2*)Vt, VTS, KW, S->r, 1, 2, R, eP1, EX, st));
            const int rcap = rmax < KW ? rmax : KW;   // a rank never exceeds the basis width
            OzSliceArgs s1;
            memset(&s1, 0, sizeof(s1));
            s1.S = 4;
            s1.X[0] = Vw;
            s1.rs[0] = 1;
            s1.cs[0] = KW;
            s1.rows[0] = rcap;
            s1.drows[0] = &S->r[0];
            s1.K[0] = R;
            s1.kscale[0] = xin;
            s1.planes[0] = pP2;
            s1.exps[0] = eP2;
            s1.tiles_k[0] = p.tkC;
            s1.tile_h[0] = OZ_CORE_NT;
            STAGE("core_prep", launch_oz_slice(s1, 1, st));
            OzBatch ob;
            memset(&ob, 0, sizeof(ob));
            ob.nbatch = 1;
            ob.err = ozerr;
            OzProblem& q = ob.p[0];
            q.kr = OzKR{(const float2*)(Vt + VTS), (const float2*)(Vt + 2 * VTS), KW, eP1 + EX, eP1 + 2 * EX};
            q.M = rcap * rcap;
            q.M_from_r2r3 = 1;
            q.dNa = &S->r[1];
            q.dNb = &S->r[2];
            q.B = OzPlanes{pP2, 0, 0, eP2, 0, p.tkC, OZ_CORE_NT};
            q.N = rcap;
            q.dN = &S->r[0];
            q.K = R;
            q.C = beta_out;
            q.crs = -1;
            q.ccs = 1;
            // split-K by the ranks (on the device): few output tiles (small ranks) with a long
            // R spread over more SMs, the partials in the tensor-core partial buffer
            constexpr int CORE_SMAX = 8;
            const long long sstride = p.ozpart_n / CORE_SMAX;
            STAGE("core_prep", launch_core_split(S->r, R, CORE_SMAX, sstride, &S->core_split, st));
            ob.nsplit = CORE_SMAX;
            q.Cpart = ozpart;
            q.split_stride = sstride;
            q.dsplit = &S->core_split;
            STAGE("core", launch_ozgemm(ob, OZ_CORE, st));
        } else {
            STAGE("core", launch_gemm(gc, st));
        }
    }
    return RHOSVD_OK;
}

// FP32 outputs, when asked for
int Reduction::to_fp32()
{
    if (p.out_fp32) {
        // round Z (every column, zeros included) and the packed core once into the FP32 outputs
        const double* src[4] = {Zout[0], Zout[1], Zout[2], beta_out};
        float* dst[4] = {(float*)out->Z[0], (float*)out->Z[1], (float*)out->Z[2], (float*)out->beta};
        long long cnt[4] = {(long long)p.n[0] * rmax, (long long)p.n[1] * rmax, (long long)p.n[2] * rmax,
                            R > 0 ? -1 : 0};
        STAGE("copy_out", launch_to_f32(src, dst, cnt, S->r, 4, st));
    }
    return RHOSVD_OK;
}

int Reduction::run()
{
    // the path's stages in order
    int (Reduction::*const stages[])() = {
        &Reduction::reset,          &Reduction::normalise,  &Reduction::direct_bases, &Reduction::slice_sketch_operand,
        &Reduction::sketch,         &Reduction::range_basis, &Reduction::project,     &Reduction::eigen,
        &Reduction::bases_residual, &Reduction::rank_final, &Reduction::als,          &Reduction::outputs_core,
        &Reduction::to_fp32};
    for (auto f : stages) {
        const int e = (this->*f)();
        if (e) return e;
    }
    return RHOSVD_OK;
}

}  // namespace

static int c2t_impl(const rhosvd_cp* cp, const rhosvd_opts* opts, const StartBasis* sb0, const rhosvd_tucker* out,
                    void* workspace, size_t workspace_bytes, void* stream, const HadSrc* had = nullptr,
                    int als_sweeps = 0)
{
    Reduction c;
    Plan& p = c.p;
    int rc = make_plan(cp, opts, &p, sb0 ? sb0->k0 : 0, als_sweeps);
    if (rc) return rc;
    if (!out || !out->info || !out->beta) return RHOSVD_ERR_INVALID_ARG;
    for (int l = 0; l < 3; ++l) {
        if (!out->Z[l] || !out->sigma[l]) return RHOSVD_ERR_INVALID_ARG;
        if (cp->R > 0 && !cp->U[l]) return RHOSVD_ERR_INVALID_ARG;
    }
    if (cp->R > 0 && !cp->xi) return RHOSVD_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < p.total || ((uintptr_t)workspace % ALIGN) != 0)
        return RHOSVD_ERR_WORKSPACE;
    c.cp = cp;
    c.opts = opts;
    c.sb0 = sb0;
    c.out = out;
    c.had = had;
    c.bind(workspace, stream);
    return c.run();
}

extern "C" int rhosvd_c2t(const rhosvd_cp* cp, const rhosvd_opts* opts, const rhosvd_tucker* out,
                          void* workspace, size_t workspace_bytes, void* stream)
{
    return c2t_impl(cp, opts, nullptr, out, workspace, workspace_bytes, stream);
}

// The virtual canonical tensor of the product a (.) b: a's columns with rank Ra Rb (its
// columns are never read past Ra; the product source supplies every term).
static int had_view(const rhosvd_cp* a, const rhosvd_cp* b, rhosvd_cp* v)
{
    if (!a || !b || a->R < 0 || b->R < 0) return RHOSVD_ERR_INVALID_ARG;
    if ((long long)a->R * b->R > 0x7fffffffLL) return RHOSVD_ERR_INVALID_ARG;
    for (int l = 0; l < 3; ++l) {
        if (a->n[l] != b->n[l] || b->ld[l] < b->n[l]) return RHOSVD_ERR_INVALID_ARG;
        if (a->R > 0 && b->R > 0 && (!a->U[l] || !b->U[l])) return RHOSVD_ERR_INVALID_ARG;
    }
    if (a->R > 0 && b->R > 0 && (!a->xi || !b->xi)) return RHOSVD_ERR_INVALID_ARG;
    *v = *a;
    v->R = a->R * b->R;
    return RHOSVD_OK;
}

extern "C" size_t rhosvd_c2t_hadamard_workspace_size(const rhosvd_cp* a, const rhosvd_cp* b,
                                                     const rhosvd_opts* opts)
{
    rhosvd_cp v;
    if (had_view(a, b, &v) != RHOSVD_OK) return 0;
    return rhosvd_c2t_workspace_size(&v, opts);
}

extern "C" int rhosvd_c2t_hadamard(const rhosvd_cp* a, const rhosvd_cp* b, const rhosvd_opts* opts,
                                   const rhosvd_tucker* out, void* workspace, size_t workspace_bytes, void* stream)
{
    rhosvd_cp v;
    int rc = had_view(a, b, &v);
    if (rc) return rc;
    HadSrc h;
    h.b = b;
    h.Ra = a->R;
    h.xa = a->xi;
    return c2t_impl(&v, opts, nullptr, out, workspace, workspace_bytes, stream, v.R > 0 ? &h : nullptr);
}

extern "C" size_t rhosvd_c2t_als_workspace_size(const rhosvd_cp* cp, const rhosvd_opts* opts, int sweeps)
{
    Plan p;
    if (sweeps < 0 || sweeps > RHOSVD_ALS_MAX_SWEEPS || make_plan(cp, opts, &p, 0, sweeps) != RHOSVD_OK) return 0;
    return p.total;
}

extern "C" int rhosvd_c2t_als(const rhosvd_cp* cp, const rhosvd_opts* opts, int sweeps, const rhosvd_tucker* out,
                              double* energy, void* workspace, size_t workspace_bytes, void* stream)
{
    if (sweeps < 0 || sweeps > RHOSVD_ALS_MAX_SWEEPS) return RHOSVD_ERR_INVALID_ARG;
    int rc = c2t_impl(cp, opts, nullptr, out, workspace, workspace_bytes, stream, nullptr, sweeps);
    if (rc || !energy || sweeps == 0) return rc;
    Plan p;
    if (make_plan(cp, opts, &p, 0, sweeps) != RHOSVD_OK) return RHOSVD_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(energy, (char*)workspace + p.o_als_e, sizeof(double) * 6 * (size_t)sweeps,
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return RHOSVD_ERR_CUDA;
    return RHOSVD_OK;
}

extern "C" size_t rhosvd_c2t_start_workspace_size(const rhosvd_cp* cp, const rhosvd_opts* opts, int k0)
{
    Plan p;
    if (k0 < 1 || make_plan(cp, opts, &p, k0) != RHOSVD_OK) return 0;
    return p.total;
}

extern "C" int rhosvd_c2t_start(const rhosvd_cp* cp, const rhosvd_opts* opts, const double* const Q0[3],
                                const int ld[3], int k0, int iters, const rhosvd_tucker* out, void* workspace,
                                size_t workspace_bytes, void* stream)
{
    if (!cp || !Q0 || !ld || k0 < 1 || iters < 0 || iters > 1) return RHOSVD_ERR_INVALID_ARG;
    StartBasis sb;
    for (int l = 0; l < 3; ++l) {
        if (!Q0[l] || ld[l] < cp->n[l]) return RHOSVD_ERR_INVALID_ARG;
        sb.Q0[l] = Q0[l];
        sb.ld[l] = ld[l];
    }
    sb.k0 = k0;
    sb.iters = iters;
    return c2t_impl(cp, opts, &sb, out, workspace, workspace_bytes, stream);
}

extern "C" int rhosvd_cp_hadamard(const rhosvd_cp* a, const rhosvd_cp* b, double* const U_out[3],
                                  const int ld_out[3], double* xi_out, void* stream)
{
    if (!a || !b || !U_out || !ld_out || !xi_out) return RHOSVD_ERR_INVALID_ARG;
    if (a->R < 0 || b->R < 0) return RHOSVD_ERR_INVALID_ARG;
    if ((long long)a->R * b->R > 0x7fffffffLL) return RHOSVD_ERR_INVALID_ARG;
    HadArgs h;
    for (int l = 0; l < 3; ++l) {
        if (a->n[l] != b->n[l] || a->n[l] < 1 || a->ld[l] < a->n[l] || b->ld[l] < b->n[l] ||
            ld_out[l] < a->n[l] || !U_out[l])
            return RHOSVD_ERR_INVALID_ARG;
        if ((a->R > 0 && !a->U[l]) || (b->R > 0 && !b->U[l])) return RHOSVD_ERR_INVALID_ARG;
        h.A[l] = a->U[l]; h.lda[l] = a->ld[l];
        h.B[l] = b->U[l]; h.ldb[l] = b->ld[l];
        h.C[l] = U_out[l]; h.ldc[l] = ld_out[l];
        h.n[l] = a->n[l];
    }
    h.Ra = a->R;
    h.Rb = b->R;
    h.xa = a->xi;
    h.xb = b->xi;
    h.xc = xi_out;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = 0;
    STAGE("hadamard", launch_hadamard(h, st));
    return RHOSVD_OK;
}

extern "C" int rhosvd_cp_sum(double alpha, const rhosvd_cp* a, double beta, const rhosvd_cp* b,
                             double* const U_out[3], const int ld_out[3], double* xi_out, void* stream)
{
    if (!a || !b || !U_out || !ld_out || !xi_out) return RHOSVD_ERR_INVALID_ARG;
    if (a->R < 0 || b->R < 0) return RHOSVD_ERR_INVALID_ARG;
    SumArgs s;
    for (int l = 0; l < 3; ++l) {
        if (a->n[l] != b->n[l] || a->n[l] < 1 || a->ld[l] < a->n[l] || b->ld[l] < b->n[l] ||
            ld_out[l] < a->n[l] || !U_out[l])
            return RHOSVD_ERR_INVALID_ARG;
        if ((a->R > 0 && !a->U[l]) || (b->R > 0 && !b->U[l])) return RHOSVD_ERR_INVALID_ARG;
        s.A[l] = a->U[l]; s.lda[l] = a->ld[l];
        s.B[l] = b->U[l]; s.ldb[l] = b->ld[l];
        s.C[l] = U_out[l]; s.ldc[l] = ld_out[l];
        s.n[l] = a->n[l];
    }
    s.Ra = a->R;
    s.Rb = b->R;
    s.xa = a->xi;
    s.xb = b->xi;
    s.xc = xi_out;
    s.alpha = alpha;
    s.beta = beta;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = 0;
    STAGE("cp_sum", launch_cpsum(s, st));
    return RHOSVD_OK;
}

// Host side of the AA-QAOA C ABI (include/aaqaoa.h): input validation, plans,
// workspace layout, TMA tensor maps and the order of kernel launches.
//
// Pass schedule for n above the tile size (T = 13 qubits for C64, 12 for C128):
//   forward, layer l = 1..p:  low pass (cost phase T_l[C(x)] then butterflies
//     on qubits 0..T-1), then high passes of 9 qubits each; the last pass of
//     layer p folds in the reduction (and, for the gradient, lambda = O psi).
//   adjoint, layer l = p..1:  the same passes on (phi, lambda) in reverse
//     order with the inverse mixer, accumulating 2 Im <lambda|X_q|phi>; the
//     last pass of the layer adds 2 Im <lambda|C|phi> and applies the inverse
//     cost phase (skipped, with the store, for l = 1).
// For n <= T one CTA per parameter point runs the whole circuit in shared
// memory.
#include <cudaTypedefs.h>

#include <array>
#include <functional>
#include <tuple>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "aaqaoa.h"
#include "aaqaoa_internal.h"

using namespace aaq;

namespace {

thread_local std::string g_detail;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_detail = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(AAQAOA_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(call)                                      \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess)                        \
            return cuda_fail(e_, #call);              \
    } while (0)

#define CKL(code, what)                                          \
    do {                                                         \
        int c_ = (code);                                         \
        if (c_ != 0)                                             \
            return cuda_fail((cudaError_t)c_, what);             \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

constexpr int MAX_PASSES = 8;  // passes per layer (tensor maps kept per pass)

struct Pass {
    int s;       // first qubit of the tile rows
    int cb;      // contiguous bits per row
    int is_low;  // contiguous tile whose low qubits are transformed
    int hmask;   // high local bits that receive a butterfly
    int wide;    // tensor-map form (rows of more than 128 bytes)
    int skip_last = 0;  // low pass done after register stage 1
    int qubits = 0;     // butterflies of this pass
    int cluster = 0;    // the 14-qubit low pass of a cluster of 4 CTAs (complex64 adjoint)
};

struct Layout {
    size_t ctrl, out, params, cs, tab, partials, zz, samp, ising, phi, lam, total;
    size_t partial_count;
};

}  // namespace

struct aaqaoa_plan {
    int n = 0, m = 0, p = 0, num_orbits = 0;
    bool c128 = false;
    std::vector<int32_t> edges;  // normalised (u < v), caller's edge order
    std::vector<int32_t> orbit_rep, orbit_weight;
    std::vector<int32_t> edge_orbit;  // class of every edge (empty when the caller gave none)
    std::vector<int32_t> edge_w;      // integer edge weights (all 1 for MaxCut)
    int wsum = 0;                     // sum of the edge weights: the largest cut value
    CostFn cost{};
    CutFn obs[2]{};
    // Ising plans (aaqaoa_prepare_ising): real couplings and fields; the
    // cost and both observables as dense functions, copied into the workspace
    bool ising = false;
    std::vector<double> ising_w, ising_h;   // per edge; per vertex (empty: no fields)
    std::vector<int32_t> vorbit_rep, vorbit_weight;
    std::vector<IsingFn> ifn;               // Ising plans: cost, H_C, H_red (1.1 MB; empty otherwise)
    const double *cur_gamma = nullptr;      // device gamma of the call being enqueued
    cudaStream_t stream = nullptr;
    // workspace
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    int cap = 0;
    bool ws_grad = false;
    Layout L{};
    std::vector<Pass> passes;      // forward passes (one-vector tile geometry)
    std::vector<Pass> bwd_passes;  // adjoint passes (two-vector tile geometry)
    std::vector<CUtensorMap> map_phi;            // forward, per pass
    std::vector<CUtensorMap> map_bphi, map_blam; // adjoint, per pass
    std::vector<std::array<CUtensorMap, 4>> map_bcl;  // cluster passes: load phi, lambda; store phi, lambda
    int launches = 0;
    bool state_valid = false;
    int inject = 0;  // pending test fault (aaqaoa_inject_fault)
    // launch profiling
    bool prof = false;
    struct ProfRec {
        int kind;
        int flags;  // bit 0: cut-function work, bit 1: fused layer boundary
        double bytes;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;

    int T() const { return tile_bits(c128); }
    int CB() const { int t, c, h; pass_geometry(c128, 1, &t, &c, &h); return c; }
    int HB() const { int t, c, h; pass_geometry(c128, 1, &t, &c, &h); return h; }
    size_t amp() const { return c128 ? 16 : 8; }
    int tab_len() const { return wsum + 1; }  // cut values 0..sum of edge weights
    int out_stride() const { return 1 + 2 * p; }
    bool small() const { return n <= T(); }
    int tiles() const { return small() ? 1 : 1 << (n - T()); }
    bool fuse = true;  // fuse layer boundaries into one pass where the plan allows
    int *err_shared = nullptr;  // set when the plan is part of a multi-graph batch
    const GraphFns *pt_dev = nullptr;  // set for a group of same-n graphs: point b is graph b
    int *d_err() const { return err_shared ? err_shared : reinterpret_cast<int *>(ws + L.ctrl); }
    unsigned *d_counter_pass() const { return reinterpret_cast<unsigned *>(ws + L.ctrl + 8); }
    unsigned *d_counter_agg() const { return reinterpret_cast<unsigned *>(ws + L.ctrl + 16); }
    double *d_out() const { return reinterpret_cast<double *>(ws + L.out); }
    double *d_params() const { return reinterpret_cast<double *>(ws + L.params); }
    double2 *d_cs() const { return reinterpret_cast<double2 *>(ws + L.cs); }
    void *d_tab() const { return ws + L.tab; }
    double *d_partials() const { return reinterpret_cast<double *>(ws + L.partials); }
    double *d_zz() const { return reinterpret_cast<double *>(ws + L.zz); }
    // sampling scratch: chunk masses | total | u[SMAX] | x[SMAX] | cut[SMAX]
    double *d_samp_sums() const { return reinterpret_cast<double *>(ws + L.samp); }
    double *d_samp_total() const { return d_samp_sums() + sample_chunk_count(n); }
    double *d_samp_u() const { return d_samp_total() + 32; }
    unsigned long long *d_samp_x() const { return reinterpret_cast<unsigned long long *>(d_samp_u() + AAQAOA_SAMPLE_MAX); }
    int *d_samp_cut() const { return reinterpret_cast<int *>(d_samp_x() + AAQAOA_SAMPLE_MAX); }
    unsigned long long *d_maxcut_key() const { return reinterpret_cast<unsigned long long *>(ws + L.ctrl + 32); }
    const IsingFn *d_ifn(int k) const { return reinterpret_cast<const IsingFn *>(ws + L.ising) + k; }
    void *d_phi() const { return ws + L.phi; }
    void *d_lam() const { return ws + L.lam; }
};

namespace {

enum ProfKind { PK_FWD = 0, PK_ADJ = 1, PK_SMALL = 2, PK_AGG = 3, PK_PARAMS = 4, PK_COUNT = 5 };

cudaEvent_t prof_event(aaqaoa_plan *pl)
{
    if (!pl->prof_pool.empty()) {
        cudaEvent_t e = pl->prof_pool.back();
        pl->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// brackets one launch with an event pair when profiling is on
struct ProfScope {
    aaqaoa_plan *pl;
    int kind;
    double bytes;
    int flags;
    cudaEvent_t a = nullptr;
    ProfScope(aaqaoa_plan *p, int k, double by, int fl = 0) : pl(p), kind(k), bytes(by), flags(fl)
    {
        if (pl->prof) {
            a = prof_event(pl);
            cudaEventRecord(a, pl->stream);
        }
    }
    ~ProfScope()
    {
        if (pl->prof) {
            cudaEvent_t b = prof_event(pl);
            cudaEventRecord(b, pl->stream);
            pl->prof_recs.push_back({kind, flags, bytes, a, b});
        }
    }
};

// profile flags of a tiled pass
int pass_flags(const PassArgs &a)
{
    return ((a.pre_phase || a.pre_lambda || a.post) ? 1 : 0) | (a.fuse ? 2 : 0) | ((a.post & POST_LAMBDA) ? 8 : 0);
}

Layout layout(const aaqaoa_plan *pl, int batch, bool grad)
{
    Layout L{};
    size_t off = 0;
    const size_t B = (size_t)batch;
    L.ctrl = off;
    off += 256;
    L.out = off;
    off = align256(off + B * pl->out_stride() * sizeof(double));
    L.params = off;
    off = align256(off + 2 * B * pl->p * sizeof(double));
    L.cs = off;
    off = align256(off + B * pl->p * sizeof(double2));
    L.tab = off;  // three tables: exact, forward-scaled, inverse layer
    off = align256(off + 3 * B * pl->p * pl->tab_len() * pl->amp());
    const size_t pass_partials = pl->small() ? 0 : 3 * B * (size_t)device_sms();
    const size_t agg_partials = 64 * (size_t)agg_grid(pl->c128);
    L.partial_count = pass_partials > agg_partials ? pass_partials : agg_partials;
    L.partials = off;
    off = align256(off + L.partial_count * sizeof(double));
    L.zz = off;
    off = align256(off + (size_t)(pl->m > 0 ? pl->m : 1) * sizeof(double));
    L.samp = off;
    off = align256(off + (sample_chunk_count(pl->n) + 32 + 2 * (size_t)AAQAOA_SAMPLE_MAX) * sizeof(double) +
                   (size_t)AAQAOA_SAMPLE_MAX * sizeof(int));
    L.ising = off;
    off = align256(off + (pl->ising ? 3 * sizeof(IsingFn) : 0));
    L.phi = off;
    off = align256(off + B * ((size_t)1 << pl->n) * pl->amp());
    L.lam = off;
    if (grad && !pl->small())
        off = align256(off + B * ((size_t)1 << pl->n) * pl->amp());
    L.total = off;
    return L;
}

// 5-D view of B statevectors for tiles of 2^T amplitudes: rows of 2^cb
// contiguous amplitudes along qubits s..s+T-cb-1. A 128-byte segment holds
// 2^cbmin amplitudes. Nine row qubits (cb = cbmin) need two box dimensions
// (32 x 16 rows); up to eight fit one (wide form, rows of 2^(cb-cbmin)
// segments).
int make_map(CUtensorMap *map, void *base, int n, int s, int cb, int T, int cbmin, size_t amp, int B, int *wide)
{
    auto fn = encode_fn();
    if (!fn)
        return fail(AAQAOA_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable from the driver");
    const int h = T - cb;
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5];
    if (h == 9) {
        dims[0] = 16; dims[1] = (cuuint64_t)1 << (s - cb); dims[2] = 32; dims[3] = 16;
        dims[4] = ((cuuint64_t)1 << (n - s - 9)) * (cuuint64_t)B;
        strides[0] = 128; strides[1] = ((cuuint64_t)1 << s) * amp; strides[2] = ((cuuint64_t)1 << (s + 5)) * amp;
        strides[3] = ((cuuint64_t)1 << (s + 9)) * amp;
        box[0] = 16; box[1] = 1; box[2] = 32; box[3] = 16; box[4] = 1;
        *wide = 0;
    } else if (h >= 0 && h <= 8 && cb >= cbmin) {
        dims[0] = 16; dims[1] = (cuuint64_t)1 << (cb - cbmin); dims[2] = (cuuint64_t)1 << (s - cb);
        dims[3] = (cuuint64_t)1 << h; dims[4] = ((cuuint64_t)1 << (n - s - h)) * (cuuint64_t)B;
        strides[0] = 128; strides[1] = ((cuuint64_t)1 << cb) * amp; strides[2] = ((cuuint64_t)1 << s) * amp;
        strides[3] = ((cuuint64_t)1 << (s + h)) * amp;
        box[0] = 16; box[1] = (cuuint32_t)1 << (cb - cbmin); box[2] = 1; box[3] = (cuuint32_t)1 << h; box[4] = 1;
        *wide = 1;
    } else {
        return fail(AAQAOA_ERR_UNSUPPORTED, "tile of %d row qubits", h);
    }
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(AAQAOA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for n=%d s=%d cb=%d", (int)r, n, s, cb);
    return AAQAOA_OK;
}

// The cluster low pass's views of B complex64 statevectors: 5-D
// [16 amplitudes][64 rows: qubits 4..9][qubits 10, 11][qubits 12, 13]
// [2^(n-14) B cluster tiles]. A CTA loads the box with qubits 12, 13 fixed
// (its rank) and stores the box with qubits 10, 11 fixed.
int make_cluster_map(CUtensorMap *map, void *base, int n, int B, bool load)
{
    auto fn = encode_fn();
    if (!fn)
        return fail(AAQAOA_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable from the driver");
    if (n < CLUSTER_LOW_QUBITS)
        return fail(AAQAOA_ERR_UNSUPPORTED, "cluster low pass needs n >= %d", CLUSTER_LOW_QUBITS);
    const cuuint64_t amp = 8;
    cuuint64_t dims[5] = {16, 64, 4, 4, ((cuuint64_t)1 << (n - CLUSTER_LOW_QUBITS)) * (cuuint64_t)B};
    cuuint64_t strides[4] = {16 * amp, ((cuuint64_t)1 << 10) * amp, ((cuuint64_t)1 << 12) * amp,
                             ((cuuint64_t)1 << 14) * amp};
    cuuint32_t box[5] = {16, 64, load ? 4u : 1u, load ? 1u : 4u, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(AAQAOA_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d) for the cluster pass, n=%d", (int)r, n);
    return AAQAOA_OK;
}

// Passes of one layer for tiles of T qubits: a low pass over qubits 0..L-1
// (contiguous tiles), then K high passes that share the remaining n-L qubits
// evenly. A high pass with h < hbmax row qubits spends the spare tile bits on
// longer contiguous rows (cb = T-h), which keeps the strided passes close to
// streaming bandwidth. Returns false when (L, K) does not give valid tiles.
// cluster_low: the geometry allows a low pass of CLUSTER_LOW_QUBITS qubits by
// a cluster of 4 CTAs (the complex64 two-vector tiles), chosen by L = 14.
// big_last (the adjoint's passes): the larger high groups come last, so that
// the adjoint's last group can be the forward's last, smaller one (the pair a
// turnaround pass takes).
bool layer_passes(int n, int T, int cbmin, int hbmax, int L2, int L, int K, std::vector<Pass> &v,
                  bool cluster_low = false, bool big_last = false)
{
    v.clear();
    const bool cl = cluster_low && L == CLUSTER_LOW_QUBITS && T + 2 == CLUSTER_LOW_QUBITS;
    if (n <= T || L < cbmin || (L > T && !cl) || K < 1 || n - L < K || n - L > K * hbmax || K + 1 > MAX_PASSES)
        return false;
    Pass low{cbmin, cbmin, 1, (1 << ((cl ? T : L) - cbmin)) - 1, 0};
    low.skip_last = !cl && L <= L2 && L < T ? 1 : 0;
    low.qubits = L;
    low.cluster = cl ? 1 : 0;
    v.push_back(low);
    const int r = n - L;
    int s = L;
    for (int k = 0; k < K; k++) {
        const int h = r / K + ((big_last ? k >= K - r % K : k < r % K) ? 1 : 0);
        if (h > hbmax || T - h > s || T - h < cbmin)  // contiguous bits stay below the rows
            return false;
        Pass hp{s, T - h, 0, (1 << h) - 1, 0};
        hp.qubits = h;
        v.push_back(hp);
        s += h;
    }
    return true;
}

// The default plan: the fewest high passes, K = ceil((n-T)/hbmax); the low
// pass covers T qubits unless those K passes can take all but the L2 qubits
// of its first two register stages, in which case it skips its third stage.
void default_layer(int n, int T, int cbmin, int hbmax, int L2, int *L, int *K, bool big_last = false)
{
    *K = (n - T + hbmax - 1) / hbmax;
    std::vector<Pass> v;
    *L = (L2 < T && layer_passes(n, T, cbmin, hbmax, L2, L2, *K, v, false, big_last)) ? L2 : T;
}

void build_passes(aaqaoa_plan *pl)
{
    pl->passes.clear();
    pl->bwd_passes.clear();
    if (pl->small())
        return;
    for (int nv = 1; nv <= 2; nv++) {
        int T, CB, HB, L, K;
        pass_geometry(pl->c128, nv, &T, &CB, &HB);
        const int L2 = low_two_stage_bits(pl->c128, nv);
        default_layer(pl->n, T, CB, HB, L2, &L, &K, nv == 2);
        layer_passes(pl->n, T, CB, HB, L2, L, K, nv == 1 ? pl->passes : pl->bwd_passes, false, nv == 2);
    }
}

// table `kind` (0 exact, 1 forward-scaled, 2 inverse) of a call with B points
const void *tab_kind(const aaqaoa_plan *pl, const void *base, int B, int kind)
{
    return static_cast<const unsigned char *>(base) + (size_t)kind * B * pl->p * pl->tab_len() * pl->amp();
}

PassArgs base_args(const aaqaoa_plan *pl, int obs)
{
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.n = pl->n;
    a.tiles = pl->tiles();
    a.B = 1;
    a.p = pl->p;
    a.tab_len = pl->tab_len();
    a.amp0 = std::pow(2.0, -0.5 * pl->n);
    a.tab = pl->d_tab();
    a.cs = pl->d_cs();
    a.partials = pl->d_partials();
    a.counter = pl->d_counter_pass();
    a.out = pl->d_out();
    a.out_stride = pl->out_stride();
    a.slot_idx[0] = a.slot_idx[1] = a.slot_idx[2] = -1;
    a.err = pl->d_err();
    a.obs = pl->obs[obs];
    a.cost = pl->cost;
    a.pt = pl->pt_dev;
    a.pt_obs = obs;
    if (pl->ising) {
        a.icost = pl->d_ifn(0);
        a.iobs = pl->d_ifn(1 + obs);
        a.gam = pl->cur_gamma;
    }
    return a;
}

// One launch of a layer sequence: pass k of the layer plan applied for
// `layer`; layer2 >= 0 marks a fused pass that also applies layer2's mixer to
// the same qubits (the boundary between two consecutive layers). j0 counts
// the layer's butterflies done by its earlier passes.
struct Step {
    int k, layer, layer2, j0;
    bool first_of_layer;  // first pass with this layer's own operations
    bool last_of_layer;   // the layer's mixer is complete after this pass
};

// Every layer runs its low pass first, then its high passes in order. With
// fusion (at least two high passes and two layers) the last pass of a layer
// also starts the next layer in the direction of travel on the same qubits,
// and the next layer skips that group and ends on another high group, so
// consecutive boundaries alternate between the last two high groups. The last
// pass of a layer is always a high pass (its last register stage carries the
// layer-end work). first (optional) overrides the first layer's order;
// start_skip is a group the first layer's mixer already has (the adjoint
// after a turnaround pass), its qubits counted in j0.
std::vector<Step> layer_schedule_from(int p, const std::vector<Pass> &passes, bool fuse, bool reverse,
                                      const std::vector<int> &first, int start_skip)
{
    const int np = (int)passes.size();
    fuse = fuse && np >= 3 && p >= 2;
    std::vector<Step> out;
    int skip = start_skip;                                         // group this layer already has
    int done0 = start_skip >= 0 ? passes[start_skip].qubits : 0;  // its qubits
    for (int i = 0; i < p; i++) {
        const int l = reverse ? p - 1 - i : i;
        const bool more = i + 1 < p;
        const int next = reverse ? l - 1 : l + 1;
        std::vector<int> order;
        if (i == 0 && !first.empty()) {
            order = first;
        } else {
            for (int k = 0; k < np; k++)
                if (k != skip)
                    order.push_back(k);
        }
        int j0 = done0;
        for (size_t o = 0; o < order.size(); o++) {
            const int k = order[o];
            const bool last = o + 1 == order.size();
            Step st{k, l, (fuse && more && last) ? next : -1, j0, o == 0 && skip < 0, last};
            j0 += passes[k].qubits;
            out.push_back(st);
        }
        skip = -1;
        done0 = 0;
        if (fuse && more) {
            skip = order.back();
            done0 = passes[skip].qubits;
        }
    }
    return out;
}

// The sweep's schedule. gen_high (complex64 forward sweeps): the first layer
// with two or more high passes starts on a high group, so that the pass
// generating |+>^n (no load, the first cost phase, compute-bound) covers a
// high group in two register stages rather than the low pass's three, and
// the low pass becomes a streaming one (complex128 passes are bound by FP64
// arithmetic either way, and their kernels keep generation in stage 0).
// end_k >= 0: the forward sweep must end on group end_k (the turnaround's
// group); the first layer's order is chosen for that, and an empty schedule
// says no order ends there.
std::vector<Step> layer_schedule(int p, const std::vector<Pass> &passes, bool fuse, bool reverse, bool gen_high,
                                 int end_k = -1, int start_skip = -1)
{
    const int np = (int)passes.size();
    std::vector<int> dflt;
    for (int k = 0; k < np; k++)
        if (k != start_skip)
            dflt.push_back(k);
    if (gen_high && !reverse && np >= 3 && start_skip < 0)
        std::swap(dflt[0], dflt[1]);
    if (end_k < 0)
        return layer_schedule_from(p, passes, fuse, reverse, dflt, start_skip);
    // candidate first-layer orders: the default, then the same with the two
    // high groups at its ends exchanged (the first layer's last group fixes
    // where every later layer ends)
    std::vector<std::vector<int>> cands{dflt};
    if (np >= 3) {
        std::vector<int> alt = dflt;
        const int a = gen_high ? 0 : 1;  // the first high group of the order
        std::swap(alt[a], alt.back());
        cands.push_back(alt);
    }
    for (const auto &c : cands) {
        if (passes[c.back()].is_low)
            continue;
        std::vector<Step> st = layer_schedule_from(p, passes, fuse, reverse, c, start_skip);
        if (!st.empty() && st.back().k == end_k)
            return st;
    }
    return {};
}

bool plan_fuses(const aaqaoa_plan *pl) { return pl->fuse && !pl->pt_dev; }

// The turnaround of a fused gradient evaluation: one two-vector pass takes
// the forward's last group (mixed forward on phi alone, then the energy and
// lambda = O phi of the exact final state) and the adjoint's first (both
// vectors mixed back with the dE/dbeta terms), so phi is read once and the
// final state never stored: the forward's last pass and the adjoint's first
// (5 S of traffic) become one launch (complex64: 2 S, phi is left as
// loaded, see enqueue_backward; complex128: 3 S). It needs the forward's last
// group to be one of the adjoint's high groups (same first qubit and size)
// and a forward order that ends there. kf, kb: those groups, or -1.
struct Turn {
    int kf = -1, kb = -1;
};
Turn turnaround(const aaqaoa_plan *pl)
{
    Turn t;
    // the adjoint's first layer keeps a high pass after the turnaround's group
    // (its last stage carries dE/dgamma and the inverse phase)
    if (!plan_fuses(pl) || pl->small() || pl->passes.size() < 3 || pl->bwd_passes.size() < 3)
        return t;
    for (size_t kb = 0; kb < pl->bwd_passes.size(); kb++) {
        const Pass &b = pl->bwd_passes[kb];
        if (b.is_low || b.cluster)
            continue;
        for (size_t kf = 0; kf < pl->passes.size(); kf++) {
            const Pass &f = pl->passes[kf];
            if (f.is_low || f.s != b.s || f.qubits != b.qubits)
                continue;
            if (layer_schedule(pl->p, pl->passes, true, false, !pl->c128, (int)kf).empty())
                continue;
            t.kf = (int)kf;
            t.kb = (int)kb;
            return t;
        }
    }
    return t;
}

enum FwdMode { FWD_ENERGY, FWD_GRAD, FWD_STATE };

// Arguments of launch i (of n) of a forward sweep: pass sp of the schedule
// over B points. The workspace pointers are the plan's (base_args).
PassArgs forward_args(const aaqaoa_plan *pl, int obs, int B, const Step &sp, size_t i, size_t n, FwdMode mode)
{
    const Pass &ps = pl->passes[sp.k];
    PassArgs a = base_args(pl, obs);
    a.B = B;
    a.s = ps.s;
    a.cb = ps.cb;
    a.wide_rows = ps.wide;
    a.is_low = ps.is_low;
    a.hmask = ps.hmask;
    a.skip_last = ps.skip_last;
    a.layer = sp.layer;
    a.tab_layer = sp.layer;
    a.sign_s = 1.0;
    a.tab = pl->ws ? tab_kind(pl, pl->d_tab(), B, 1) : nullptr;  // the static path sets its own
    a.load = i > 0;
    // a layer's phase comes with its first pass, or at the end of the fused
    // pass that starts it
    a.pre_phase = sp.first_of_layer ? 1 : 0;
    a.nvec_io = 1;
    const bool last = i + 1 == n;
    a.write = !(last && mode == FWD_ENERGY);
    a.post = (last && mode != FWD_STATE) ? POST_REDUCE : 0;
    if (last && a.write)
        a.post |= POST_RESCALE;
    if (last && mode != FWD_STATE) {
        a.slot_idx[0] = 0;
        a.slot_scale[0] = 1.0;
    }
    if (sp.layer2 >= 0) {
        a.fuse = 1;
        a.layer2 = sp.layer2;
        a.tab_layer = sp.layer2;
        a.post |= POST_PHASE;
    }
    return a;
}

// The forward sweep; for a gradient evaluation with a turnaround it ends
// one pass early (the turnaround applies the last group).
int enqueue_forward(aaqaoa_plan *pl, int B, int obs, FwdMode mode)
{
    const long long total = (long long)pl->tiles() * B;
    const int grid = pass_grid(total);
    const int chunk = B > 1 ? (int)((total + grid - 1) / grid) : 0;
    const Turn tn = mode == FWD_GRAD ? turnaround(pl) : Turn{};
    std::vector<Step> sched = layer_schedule(pl->p, pl->passes, plan_fuses(pl), false, !pl->c128, tn.kf);
    if (tn.kf >= 0)
        sched.pop_back();
    for (size_t i = 0; i < sched.size(); i++) {
        const Step &sp = sched[i];
        PassArgs a = forward_args(pl, obs, B, sp, i, sched.size() + (tn.kf >= 0 ? 1 : 0), mode);
        a.chunk = chunk;
        if (pl->inject == AAQAOA_FAULT_DROP_TILE && a.load) {
            a.drop_first_load = 1;
            pl->inject = 0;
        }
        const double S = (double)B * (double)((size_t)1 << pl->n) * (double)pl->amp();
        ProfScope ps_(pl, PK_FWD, S * ((a.load ? 1 : 0) + (a.write ? 1 : 0)), pass_flags(a));
        CKL(launch_pass(pl->c128, 1, pl->map_phi[sp.k], pl->map_phi[sp.k], a, grid, pl->stream), "forward pass");
        pl->launches++;
    }
    return AAQAOA_OK;
}

// adjoint passes on (phi, lambda); the first one forms lambda = O phi itself,
// or the turnaround pass does (it also finishes the forward sweep)
int enqueue_backward(aaqaoa_plan *pl, int B, int obs)
{
    int T, CB, HB;
    pass_geometry(pl->c128, 2, &T, &CB, &HB);
    const int tiles = 1 << (pl->n - T);
    const int grid = pass_grid((long long)tiles * B);
    const int chunk = B > 1 ? (int)(((long long)tiles * B + grid - 1) / grid) : 0;
    const double S = (double)B * (double)((size_t)1 << pl->n) * (double)pl->amp();
    const Turn tn = turnaround(pl);
    const int lp = pl->p - 1;  // the last layer: the adjoint's first
    if (tn.kb >= 0) {
        // load phi before the layer's last group, mix it forward (phi alone),
        // rescale, energy, lambda = O phi, mix both back: a fused pass whose
        // two layers are the same layer with opposite signs. Mixed back, phi
        // is the loaded phi times a known factor, so complex64 does not store
        // it: the kernel stores lambda times that factor instead (2 S moved,
        // not 3 S; complex128 stores both)
        const Pass &ps = pl->bwd_passes[tn.kb];
        PassArgs a = base_args(pl, obs);
        a.B = B;
        a.chunk = chunk;
        a.tiles = tiles;
        a.s = ps.s;
        a.cb = ps.cb;
        a.wide_rows = ps.wide;
        a.is_low = 0;
        a.hmask = ps.hmask;
        a.layer = a.layer2 = a.tab_layer = lp;
        a.sign_s = 1.0;
        a.sign2 = -1.0;
        a.tab = tab_kind(pl, pl->d_tab(), B, 1);
        a.j0 = pl->n - ps.qubits;
        a.load = 1;
        a.nvec_io = 1;
        a.write = 1;
        a.post = POST_REDUCE | POST_RESCALE | POST_LAMBDA;
        a.fuse = 1;
        a.slot_idx[0] = 0;  // the energy
        a.slot_scale[0] = 1.0;
        a.slot_idx[2] = 1 + pl->p + lp;  // dE/dbeta of the last layer, this group's share
        a.slot_scale[2] = 2.0;
        if (pl->inject == AAQAOA_FAULT_DROP_TILE) {
            a.drop_first_load = 1;
            pl->inject = 0;
        }
        ProfScope ps_(pl, PK_ADJ, S * (pl->c128 ? 3 : 2), pass_flags(a));
        CKL(launch_pass(pl->c128, 2, pl->map_bphi[tn.kb], pl->map_blam[tn.kb], a, grid, pl->stream), "turnaround pass");
        pl->launches++;
    }
    // Each layer runs its passes low pass first, so the cut-function work at
    // the layer's end (dE/dgamma, inverse phase) falls in a high pass and the
    // low pass can stop after two register stages.
    const std::vector<Step> sched = layer_schedule(pl->p, pl->bwd_passes, plan_fuses(pl), true, false, -1, tn.kb);
    for (size_t i = 0; i < sched.size(); i++) {
        const Step &sp = sched[i];
        const Pass &ps = pl->bwd_passes[sp.k];
        const int l = sp.layer;
        const bool first = i == 0 && tn.kb < 0;
        PassArgs a = base_args(pl, obs);
        a.B = B;
        a.chunk = chunk;
        a.tiles = tiles;
        a.s = ps.s;
        a.cb = ps.cb;
        a.wide_rows = ps.wide;
        a.is_low = ps.is_low;
        a.hmask = ps.hmask;
        a.skip_last = ps.skip_last;
        a.layer = l;
        a.tab_layer = l;
        a.sign_s = -1.0;
        a.tab = tab_kind(pl, pl->d_tab(), B, 2);
        a.j0 = sp.j0;
        a.load = 1;
        a.pre_phase = 0;
        a.pre_lambda = first ? 1 : 0;
        a.nvec_io = first ? 1 : 2;
        a.post = sp.last_of_layer ? (POST_GAMMA | (l > 0 ? POST_PHASE_CONJ : 0)) : 0;
        a.write = !(sp.last_of_layer && l == 0);
        a.slot_idx[0] = 1 + pl->p + l;
        a.slot_scale[0] = 2.0;
        if (sp.last_of_layer) {
            a.slot_idx[1] = 1 + l;
            a.slot_scale[1] = 2.0;
        }
        if (sp.layer2 >= 0) {  // the next layer (l - 1) starts on the same qubits
            a.fuse = 1;
            a.layer2 = sp.layer2;
            a.slot_idx[2] = 1 + pl->p + sp.layer2;
            a.slot_scale[2] = 2.0;
        }
        if (ps.cluster) {  // one launch per point, each over that point's cluster tiles
            for (int b = 0; b < B; b++) {
                PassArgs ab = a;
                ab.B = 1;
                ab.chunk = 0;
                ab.tile0 = b << (pl->n - CLUSTER_LOW_QUBITS);
                ab.cs = a.cs + (size_t)b * pl->p;
                ab.out = a.out + (size_t)b * pl->out_stride();
                ProfScope ps_(pl, PK_ADJ, S / B * (a.nvec_io + 2), pass_flags(a) | 4);
                CKL(launch_cluster_pass(pl->map_bcl[sp.k].data(), ab, pl->stream), "adjoint cluster pass");
                pl->launches++;
            }
            continue;
        }
        ProfScope ps_(pl, PK_ADJ, S * (a.nvec_io + (a.write ? 2 : 0)), pass_flags(a));
        CKL(launch_pass(pl->c128, 2, pl->map_bphi[sp.k], pl->map_blam[sp.k], a, grid, pl->stream), "adjoint pass");
        pl->launches++;
    }
    return AAQAOA_OK;
}

SmallArgs small_args(const aaqaoa_plan *pl, int obs, int mode, int write_state)
{
    SmallArgs s;
    memset(&s, 0, sizeof s);
    s.n = pl->n;
    s.p = pl->p;
    s.tab_len = pl->tab_len();
    s.mode = mode;
    s.write_state = write_state;
    s.amp0 = std::pow(2.0, -0.5 * pl->n);
    s.tab = pl->d_tab();
    s.cs = pl->d_cs();
    s.out = pl->d_out();
    s.out_stride = pl->out_stride();
    s.state = pl->d_phi();
    s.obs = pl->obs[obs];
    s.cost = pl->cost;
    if (pl->ising) {
        s.icost = pl->d_ifn(0);
        s.iobs = pl->d_ifn(1 + obs);
        s.gam = pl->cur_gamma;
    }
    return s;
}

int check_ready(aaqaoa_plan *pl, int obs, bool grad, int B)
{
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    if (!pl->ws)
        return fail(AAQAOA_ERR_WORKSPACE, "no workspace set (aaqaoa_set_workspace)");
    if (obs != AAQAOA_OBS_FULL && obs != AAQAOA_OBS_RED)
        return fail(AAQAOA_ERR_INVALID_ARG, "observable %d unknown", obs);
    if (obs == AAQAOA_OBS_RED && pl->num_orbits == 0)
        return fail(AAQAOA_ERR_INVALID_ARG, "H_red requested but the plan has no edge orbits");
    if (grad && !pl->ws_grad)
        return fail(AAQAOA_ERR_WORKSPACE, "workspace was set without room for the gradient");
    if (B < 1 || B > pl->cap)
        return fail(AAQAOA_ERR_INVALID_ARG, "batch %d outside [1, %d] (workspace capacity)", B, pl->cap);
    return AAQAOA_OK;
}

// parameters already in device memory (point-major B x p)
int enqueue_params(aaqaoa_plan *pl, int B, const double *d_gamma, const double *d_beta)
{
    (void)cudaGetLastError();  // a stale error of an unrelated earlier call must not be reported here
    pl->cur_gamma = d_gamma;
    ProfScope ps_(pl, PK_PARAMS, 0.0);
    CKL(launch_params(pl->c128, B, pl->p, pl->tab_len(), pl->n, d_gamma, d_beta, pl->d_tab(), pl->d_cs(), pl->stream),
        "parameter tables");
    pl->launches++;
    CK(cudaMemsetAsync(pl->d_out(), 0, (size_t)B * pl->out_stride() * sizeof(double), pl->stream));
    return AAQAOA_OK;
}

int enqueue_aggregate(aaqaoa_plan *pl, int obs, int agg)
{
    const bool c128 = pl->c128;
    const int grid = pl->n < 10 ? 1 : agg_grid(c128);
    CK(cudaMemsetAsync(pl->d_out(), 0, sizeof(double), pl->stream));
    AggArgs a;
    memset(&a, 0, sizeof a);
    a.n = pl->n;
    a.chunks = pl->n < 10 ? 0 : ((uint64_t)1 << (pl->n - 10));
    a.state = pl->d_phi();
    a.partials = pl->d_partials();
    a.counter = pl->d_counter_agg();
    a.out_energy = pl->d_out();
    const double S = (double)((size_t)1 << pl->n) * (double)pl->amp();
    if (agg == AAQAOA_AGG_SINGLEPASS) {
        a.obs = pl->obs[obs];
        ProfScope ps_(pl, PK_AGG, S);
        CKL(launch_agg_fused(c128, a, pl->stream, grid), "single-pass aggregation");
        pl->launches++;
        return AAQAOA_OK;
    }
    // per-term passes: Eq. (agg) over all edges (H_C) or the representatives (H_red)
    const int nterms = obs == AAQAOA_OBS_FULL ? pl->m : pl->num_orbits;
    for (int t = 0; t < nterms; t++) {
        const int e = obs == AAQAOA_OBS_FULL ? t : pl->orbit_rep[t];
        a.num_terms = 1;
        a.term_u[0] = pl->edges[2 * e];
        a.term_v[0] = pl->edges[2 * e + 1];
        a.term_w[0] = obs == AAQAOA_OBS_FULL ? (double)pl->edge_w[e] : (double)pl->orbit_weight[t] * pl->edge_w[e];
        ProfScope ps_(pl, PK_AGG, S);
        CKL(launch_agg_terms(c128, a, pl->stream, grid), "per-term aggregation");
        pl->launches++;
    }
    return AAQAOA_OK;
}

int enqueue_expect(aaqaoa_plan *pl, int B, const double *d_gamma, const double *d_beta, int obs, int agg)
{
    int r = enqueue_params(pl, B, d_gamma, d_beta);
    if (r)
        return r;
    const bool materialise = agg != AAQAOA_AGG_FUSED;
    if (pl->small()) {
        SmallArgs s = small_args(pl, obs, SMALL_ENERGY, materialise ? 1 : 0);
        ProfScope ps_(pl, PK_SMALL, materialise ? (double)B * (double)((size_t)1 << pl->n) * (double)pl->amp() : 0.0);
        CKL(launch_small(pl->c128, s, B, pl->stream), "whole-circuit kernel");
        pl->launches++;
    } else {
        pl->state_valid = false;  // the passes overwrite the stored state
        r = enqueue_forward(pl, B, obs, materialise ? FWD_STATE : FWD_ENERGY);
        if (r)
            return r;
    }
    if (materialise) {
        pl->state_valid = true;
        return enqueue_aggregate(pl, obs, agg);
    }
    return AAQAOA_OK;
}

// energy and gradient of B points (rows of d_out)
int enqueue_grad(aaqaoa_plan *pl, const double *d_gamma, const double *d_beta, int obs, int B = 1)
{
    int r = enqueue_params(pl, B, d_gamma, d_beta);
    if (r)
        return r;
    if (pl->small()) {
        SmallArgs s = small_args(pl, obs, SMALL_GRAD, 0);
        ProfScope ps_(pl, PK_SMALL, 0.0);
        CKL(launch_small(pl->c128, s, B, pl->stream), "whole-circuit kernel");
        pl->launches++;
        return AAQAOA_OK;
    }
    r = enqueue_forward(pl, B, obs, FWD_GRAD);
    if (r)
        return r;
    pl->state_valid = false;
    return enqueue_backward(pl, B, obs);
}

// copy [err | pad | out rows] back and check the device error flag
int fetch_out(aaqaoa_plan *pl, int B, std::vector<double> &rows)
{
    const size_t nout = (size_t)B * pl->out_stride();
    rows.resize(nout);
    int err = 0;
    CK(cudaMemcpyAsync(&err, pl->d_err(), sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
    CK(cudaMemcpyAsync(rows.data(), pl->d_out(), nout * sizeof(double), cudaMemcpyDeviceToHost, pl->stream));
    CK(cudaStreamSynchronize(pl->stream));
    if (err) {
        cudaMemsetAsync(pl->ws + pl->L.ctrl, 0, 256, pl->stream);
        cudaStreamSynchronize(pl->stream);
        return fail(AAQAOA_ERR_TIMEOUT, "a bounded device wait expired (TMA tile never arrived)");
    }
    return AAQAOA_OK;
}

int upload_params(aaqaoa_plan *pl, int B, const double *gamma, const double *beta)
{
    if (!gamma || !beta)
        return fail(AAQAOA_ERR_INVALID_ARG, "gamma/beta is NULL");
    const size_t bytes = (size_t)B * pl->p * sizeof(double);
    double *dg = pl->d_params(), *db = pl->d_params() + (size_t)B * pl->p;
    CK(cudaMemcpyAsync(dg, gamma, bytes, cudaMemcpyHostToDevice, pl->stream));
    CK(cudaMemcpyAsync(db, beta, bytes, cudaMemcpyHostToDevice, pl->stream));
    return AAQAOA_OK;
}

CutFn make_cutfn(int n, const std::vector<std::pair<std::pair<int, int>, int>> &wedges)
{
    CutFn f;
    memset(&f, 0, sizeof f);
    std::map<int, int> cls;
    for (auto &we : wedges)
        cls.emplace(we.second, 0);
    if ((int)cls.size() <= MAXK) {
        int c = 0;
        for (auto &kv : cls) {
            kv.second = c;
            f.w[c] = kv.first;
            c++;
        }
        f.K = c;
        for (auto &we : wedges) {
            const int c2 = cls[we.second], u = we.first.first, v = we.first.second;
            f.nbr[c2][u] |= 1ull << v;
            f.nbr[c2][v] |= 1ull << u;
        }
    } else {  // binary digits of the weights (all < 2^10 because they sum to |E| <= 561)
        f.K = MAXK;
        for (int bit = 0; bit < MAXK; bit++)
            f.w[bit] = 1 << bit;
        for (auto &we : wedges)
            for (int bit = 0; bit < MAXK; bit++)
                if ((we.second >> bit) & 1) {
                    f.nbr[bit][we.first.first] |= 1ull << we.first.second;
                    f.nbr[bit][we.first.second] |= 1ull << we.first.first;
                }
    }
    (void)n;
    return f;
}

}  // namespace

// ================================================================== ABI
extern "C" {

const char *aaqaoa_strerror(int code)
{
    switch (code) {
    case AAQAOA_OK: return "success";
    case AAQAOA_ERR_INVALID_ARG: return "invalid argument";
    case AAQAOA_ERR_BAD_ORBITS: return "edge-orbit data do not partition the edge set";
    case AAQAOA_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case AAQAOA_ERR_CUDA: return "CUDA error";
    case AAQAOA_ERR_TIMEOUT: return "bounded device wait expired";
    case AAQAOA_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown error code";
    }
}

const char *aaqaoa_last_error_detail(void) { return g_detail.c_str(); }

int aaqaoa_prepare(int n, int num_edges, const int32_t *edges, int num_orbits, const int32_t *orbit_rep,
                   const int32_t *orbit_weight, const int32_t *edge_orbit, int p, unsigned flags, void *stream,
                   aaqaoa_plan **out)
{
    return aaqaoa_prepare_weighted(n, num_edges, edges, nullptr, num_orbits, orbit_rep, orbit_weight, edge_orbit, p,
                                   flags, stream, out);
}

int aaqaoa_prepare_weighted(int n, int num_edges, const int32_t *edges, const int32_t *edge_weight, int num_orbits,
                            const int32_t *orbit_rep, const int32_t *orbit_weight, const int32_t *edge_orbit, int p,
                            unsigned flags, void *stream, aaqaoa_plan **out)
{
    g_detail.clear();
    if (!out)
        return fail(AAQAOA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > AAQAOA_MAX_QUBITS)
        return fail(AAQAOA_ERR_INVALID_ARG, "n=%d outside [1, %d]", n, AAQAOA_MAX_QUBITS);
    if (p < 1 || p > 64)
        return fail(AAQAOA_ERR_INVALID_ARG, "p=%d outside [1, 64]", p);
    if (flags != AAQAOA_C64 && flags != AAQAOA_C128)
        return fail(AAQAOA_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
    if (num_edges < 0 || (long long)num_edges > (long long)n * (n - 1) / 2)
        return fail(AAQAOA_ERR_INVALID_ARG, "num_edges=%d impossible for n=%d", num_edges, n);
    if (num_edges > 0 && !edges)
        return fail(AAQAOA_ERR_INVALID_ARG, "edges is NULL");
    std::vector<int32_t> e(2 * (size_t)num_edges);
    uint64_t adj[AAQAOA_MAX_QUBITS] = {0};
    for (int i = 0; i < num_edges; i++) {
        int u = edges[2 * i], v = edges[2 * i + 1];
        if (u < 0 || u >= n || v < 0 || v >= n)
            return fail(AAQAOA_ERR_INVALID_ARG, "edge %d = (%d, %d) has a vertex outside [0, %d)", i, u, v, n);
        if (u == v)
            return fail(AAQAOA_ERR_INVALID_ARG, "edge %d is a self-loop on %d", i, u);
        if (u > v)
            std::swap(u, v);
        if ((adj[u] >> v) & 1ull)
            return fail(AAQAOA_ERR_INVALID_ARG, "edge %d = (%d, %d) is repeated", i, u, v);
        adj[u] |= 1ull << v;
        adj[v] |= 1ull << u;
        e[2 * i] = u;
        e[2 * i + 1] = v;
    }
    std::vector<int32_t> w(num_edges, 1);
    long long wsum = 0;
    for (int i = 0; i < num_edges; i++) {
        if (edge_weight) {
            if (edge_weight[i] < 1)
                return fail(AAQAOA_ERR_INVALID_ARG, "edge %d has weight %d < 1", i, edge_weight[i]);
            w[i] = edge_weight[i];
        }
        wsum += w[i];
    }
    if (wsum > MAXTAB - 1)
        return fail(AAQAOA_ERR_UNSUPPORTED, "total edge weight %lld exceeds the phase-table limit %d", wsum,
                    MAXTAB - 1);
    if (num_orbits < 0)
        return fail(AAQAOA_ERR_BAD_ORBITS, "num_orbits=%d < 0", num_orbits);
    if (num_orbits > 0) {
        if (!orbit_rep || !orbit_weight)
            return fail(AAQAOA_ERR_BAD_ORBITS, "orbit_rep / orbit_weight is NULL");
        if (num_orbits > num_edges)
            return fail(AAQAOA_ERR_BAD_ORBITS, "more orbits (%d) than edges (%d)", num_orbits, num_edges);
        long long sum = 0;
        std::vector<char> isrep(num_edges, 0);
        for (int c = 0; c < num_orbits; c++) {
            if (orbit_rep[c] < 0 || orbit_rep[c] >= num_edges)
                return fail(AAQAOA_ERR_BAD_ORBITS, "orbit %d representative %d is not an edge index", c, orbit_rep[c]);
            if (isrep[orbit_rep[c]])
                return fail(AAQAOA_ERR_BAD_ORBITS, "edge %d represents two orbits", orbit_rep[c]);
            isrep[orbit_rep[c]] = 1;
            if (orbit_weight[c] < 1)
                return fail(AAQAOA_ERR_BAD_ORBITS, "orbit %d has weight %d < 1", c, orbit_weight[c]);
            sum += orbit_weight[c];
        }
        if (sum != num_edges)
            return fail(AAQAOA_ERR_BAD_ORBITS, "orbit weights sum to %lld, not |E| = %d", sum, num_edges);
        if (edge_orbit) {
            std::vector<int> count(num_orbits, 0);
            for (int i = 0; i < num_edges; i++) {
                if (edge_orbit[i] < 0 || edge_orbit[i] >= num_orbits)
                    return fail(AAQAOA_ERR_BAD_ORBITS, "edge %d has orbit %d outside [0, %d)", i, edge_orbit[i],
                                num_orbits);
                count[edge_orbit[i]]++;
            }
            for (int c = 0; c < num_orbits; c++) {
                if (edge_orbit[orbit_rep[c]] != c)
                    return fail(AAQAOA_ERR_BAD_ORBITS, "representative of orbit %d lies in orbit %d", c,
                                edge_orbit[orbit_rep[c]]);
                if (count[c] != orbit_weight[c])
                    return fail(AAQAOA_ERR_BAD_ORBITS, "orbit %d has %d edges but weight %d", c, count[c],
                                orbit_weight[c]);
            }
            for (int i = 0; i < num_edges; i++)  // automorphisms of a weighted graph keep edge weights
                if (w[i] != w[orbit_rep[edge_orbit[i]]])
                    return fail(AAQAOA_ERR_BAD_ORBITS, "orbit %d mixes edge weights %d and %d", edge_orbit[i], w[i],
                                w[orbit_rep[edge_orbit[i]]]);
        }
    } else if (edge_orbit) {
        return fail(AAQAOA_ERR_BAD_ORBITS, "edge_orbit given without orbits");
    }

    aaqaoa_plan *pl = new (std::nothrow) aaqaoa_plan();
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "out of host memory");
    pl->n = n;
    pl->m = num_edges;
    pl->p = p;
    pl->num_orbits = num_orbits;
    pl->c128 = (flags == AAQAOA_C128);
    pl->edges = e;
    pl->orbit_rep.assign(orbit_rep, orbit_rep + num_orbits);
    pl->orbit_weight.assign(orbit_weight, orbit_weight + num_orbits);
    if (edge_orbit)
        pl->edge_orbit.assign(edge_orbit, edge_orbit + num_edges);
    pl->stream = (cudaStream_t)stream;
    pl->edge_w = w;
    pl->wsum = (int)wsum;
    std::vector<std::pair<std::pair<int, int>, int>> full, red;
    for (int i = 0; i < num_edges; i++)
        full.push_back({{e[2 * i], e[2 * i + 1]}, w[i]});
    for (int c = 0; c < num_orbits; c++) {
        const int i = orbit_rep[c];
        red.push_back({{e[2 * i], e[2 * i + 1]}, orbit_weight[c] * w[i]});
    }
    pl->cost = make_cutfn(n, full);
    pl->obs[AAQAOA_OBS_FULL] = make_cutfn(n, full);
    pl->obs[AAQAOA_OBS_RED] = make_cutfn(n, red);
    build_passes(pl);
    *out = pl;
    return AAQAOA_OK;
}

int aaqaoa_prepare_ising(int n, int num_edges, const int32_t *edges, const double *edge_weight, const double *field,
                         int num_orbits, const int32_t *orbit_rep, const int32_t *orbit_weight,
                         const int32_t *edge_orbit, int num_vorbits, const int32_t *vorbit_rep,
                         const int32_t *vorbit_weight, const int32_t *vertex_orbit, int p, unsigned flags, void *stream,
                         aaqaoa_plan **out)
{
    // edges, p, flags and the edge-orbit partition are checked as for MaxCut
    aaqaoa_plan *pl = nullptr;
    int r = aaqaoa_prepare_weighted(n, num_edges, edges, nullptr, num_orbits, orbit_rep, orbit_weight, edge_orbit, p,
                                    flags, stream, &pl);
    if (r)
        return r;
    *out = nullptr;
    auto reject = [&](int code, const char *fmt, auto... args) {
        aaqaoa_destroy(pl);
        return fail(code, fmt, args...);
    };
    if (num_edges > 0 && !edge_weight)
        return reject(AAQAOA_ERR_INVALID_ARG, "edge_weight is NULL (%d edges)", num_edges);
    for (int i = 0; i < num_edges; i++)
        if (!std::isfinite(edge_weight[i]))
            return reject(AAQAOA_ERR_INVALID_ARG, "edge %d has a weight that is not finite", i);
    if (field)
        for (int u = 0; u < n; u++)
            if (!std::isfinite(field[u]))
                return reject(AAQAOA_ERR_INVALID_ARG, "vertex %d has a field that is not finite", u);
    if (edge_orbit)  // automorphisms keep the couplings: one weight per class
        for (int i = 0; i < num_edges; i++)
            if (edge_weight[i] != edge_weight[orbit_rep[edge_orbit[i]]])
                return reject(AAQAOA_ERR_BAD_ORBITS, "orbit %d mixes edge weights (edge %d)", edge_orbit[i], i);
    // vertex orbits: needed for H_red when there are fields
    if (num_vorbits < 0 || num_vorbits > n)
        return reject(AAQAOA_ERR_BAD_ORBITS, "num_vorbits=%d outside [0, n=%d]", num_vorbits, n);
    if (field && num_orbits > 0 && num_vorbits == 0)
        return reject(AAQAOA_ERR_BAD_ORBITS, "fields with edge orbits need vertex orbits for H_red");
    if (num_vorbits > 0) {
        if (!vorbit_rep || !vorbit_weight)
            return reject(AAQAOA_ERR_BAD_ORBITS, "vorbit_rep / vorbit_weight is NULL");
        std::vector<char> isrep(n, 0);
        long long sum = 0;
        for (int c = 0; c < num_vorbits; c++) {
            if (vorbit_rep[c] < 0 || vorbit_rep[c] >= n)
                return reject(AAQAOA_ERR_BAD_ORBITS, "vertex orbit %d representative %d is not a vertex", c,
                              vorbit_rep[c]);
            if (isrep[vorbit_rep[c]])
                return reject(AAQAOA_ERR_BAD_ORBITS, "vertex %d represents two orbits", vorbit_rep[c]);
            isrep[vorbit_rep[c]] = 1;
            if (vorbit_weight[c] < 1)
                return reject(AAQAOA_ERR_BAD_ORBITS, "vertex orbit %d has weight %d < 1", c, vorbit_weight[c]);
            sum += vorbit_weight[c];
        }
        if (sum != n)
            return reject(AAQAOA_ERR_BAD_ORBITS, "vertex orbit weights sum to %d, not n = %d", (int)sum, n);
        if (vertex_orbit) {
            std::vector<int> count(num_vorbits, 0);
            for (int u = 0; u < n; u++) {
                if (vertex_orbit[u] < 0 || vertex_orbit[u] >= num_vorbits)
                    return reject(AAQAOA_ERR_BAD_ORBITS, "vertex %d has orbit %d out of range", u, vertex_orbit[u]);
                count[vertex_orbit[u]]++;
            }
            for (int c = 0; c < num_vorbits; c++) {
                if (vertex_orbit[vorbit_rep[c]] != c)
                    return reject(AAQAOA_ERR_BAD_ORBITS, "representative of vertex orbit %d lies in orbit %d", c,
                                  vertex_orbit[vorbit_rep[c]]);
                if (count[c] != vorbit_weight[c])
                    return reject(AAQAOA_ERR_BAD_ORBITS, "vertex orbit %d has %d vertices, not its weight %d", c, count[c], vorbit_weight[c]);
            }
            if (field)  // automorphisms keep the fields
                for (int u = 0; u < n; u++)
                    if (field[u] != field[vorbit_rep[vertex_orbit[u]]])
                        return reject(AAQAOA_ERR_BAD_ORBITS, "vertex orbit %d mixes fields (vertex %d)",
                                      vertex_orbit[u], u);
        }
    }
    pl->ising = true;
    pl->wsum = 0;  // the phase tables carry only the butterfly scale (one entry)
    pl->ising_w.assign(edge_weight, edge_weight + num_edges);
    if (field)
        pl->ising_h.assign(field, field + n);
    pl->vorbit_rep.assign(vorbit_rep, vorbit_rep + num_vorbits);
    pl->vorbit_weight.assign(vorbit_weight, vorbit_weight + num_vorbits);
    pl->ifn.clear();
    pl->ifn.resize(3);  // zeroed in place (no 1.1 MB temporary)
    for (int i = 0; i < num_edges; i++) {
        const int u = pl->edges[2 * i], v = pl->edges[2 * i + 1];
        pl->ifn[0].W[u][v] = pl->ifn[0].W[v][u] = edge_weight[i];
    }
    if (field)
        for (int u = 0; u < n; u++)
            pl->ifn[0].h[u] = field[u];
    pl->ifn[1] = pl->ifn[0];  // H_C: the cost itself
    for (int c = 0; c < num_orbits; c++) {  // H_red: representatives at orbit size x weight
        const int i = orbit_rep[c], u = pl->edges[2 * i], v = pl->edges[2 * i + 1];
        pl->ifn[2].W[u][v] = pl->ifn[2].W[v][u] = orbit_weight[c] * edge_weight[i];
    }
    if (field)
        for (int c = 0; c < num_vorbits; c++)
            pl->ifn[2].h[vorbit_rep[c]] = vorbit_weight[c] * field[vorbit_rep[c]];
    for (IsingFn &F : pl->ifn)  // chunk sums of the couplings, in FP64
        for (int c = 0; c < ISING_CHUNKS; c++)
            for (int m = 0; m < 64; m++)
                for (int u = 0; u < MAXN; u++) {
                    double g = 0.0;
                    for (int j = 0; j < 6 && 6 * c + j < MAXN; j++)
                        if ((m >> j) & 1)
                            g += F.W[6 * c + j][u];
                    F.G[c][m][u] = g;
                }
    *out = pl;
    return AAQAOA_OK;
}

int aaqaoa_workspace_bytes(const aaqaoa_plan *plan, int batch, int with_grad, size_t *bytes)
{
    if (!plan || !bytes || batch < 1)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan/bytes NULL or batch < 1");
    *bytes = layout(plan, batch, with_grad != 0).total;
    return AAQAOA_OK;
}

// TMA tensor maps of the current pass plans over the workspace's vectors
int build_maps(aaqaoa_plan *pl)
{
    pl->map_phi.assign(pl->passes.size(), CUtensorMap{});
    pl->map_bphi.assign(pl->bwd_passes.size(), CUtensorMap{});
    pl->map_blam.assign(pl->bwd_passes.size(), CUtensorMap{});
    pl->map_bcl.assign(pl->bwd_passes.size(), std::array<CUtensorMap, 4>{});
    if (!pl->ws)
        return AAQAOA_OK;
    int T, CB, HB;
    pass_geometry(pl->c128, 1, &T, &CB, &HB);
    for (size_t k = 0; k < pl->passes.size(); k++) {
        Pass &ps = pl->passes[k];
        int r = make_map(&pl->map_phi[k], pl->d_phi(), pl->n, ps.s, ps.cb, T, CB, pl->amp(), pl->cap, &ps.wide);
        if (r)
            return r;
    }
    if (pl->ws_grad) {
        pass_geometry(pl->c128, 2, &T, &CB, &HB);
        for (size_t k = 0; k < pl->bwd_passes.size(); k++) {
            Pass &ps = pl->bwd_passes[k];
            if (ps.cluster) {
                for (int j = 0; j < 4; j++) {
                    int r = make_cluster_map(&pl->map_bcl[k][j], j % 2 ? pl->d_lam() : pl->d_phi(), pl->n, pl->cap,
                                             j < 2);
                    if (r)
                        return r;
                }
                continue;
            }
            int r = make_map(&pl->map_bphi[k], pl->d_phi(), pl->n, ps.s, ps.cb, T, CB, pl->amp(), pl->cap, &ps.wide);
            if (r)
                return r;
            r = make_map(&pl->map_blam[k], pl->d_lam(), pl->n, ps.s, ps.cb, T, CB, pl->amp(), pl->cap, &ps.wide);
            if (r)
                return r;
        }
    }
    return AAQAOA_OK;
}

int aaqaoa_set_workspace(aaqaoa_plan *pl, void *device_ptr, size_t bytes, int batch, int with_grad)
{
    if (!pl || batch < 1)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan NULL or batch < 1");
    if (!device_ptr || ((uintptr_t)device_ptr & 255))
        return fail(AAQAOA_ERR_WORKSPACE, "workspace pointer NULL or not 256-byte aligned");
    Layout L = layout(pl, batch, with_grad != 0);
    if (bytes < L.total)
        return fail(AAQAOA_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", bytes, L.total);
    pl->ws = (unsigned char *)device_ptr;
    pl->ws_bytes = bytes;
    pl->cap = batch;
    pl->ws_grad = with_grad != 0;
    pl->L = L;
    pl->state_valid = false;
    int r = build_maps(pl);
    if (r)
        return r;
    CK(cudaMemsetAsync(pl->ws + L.ctrl, 0, 256, pl->stream));
    if (pl->ising)
        CK(cudaMemcpyAsync(pl->ws + L.ising, pl->ifn.data(), pl->ifn.size() * sizeof(IsingFn), cudaMemcpyHostToDevice,
                           pl->stream));
    CK(cudaStreamSynchronize(pl->stream));
    return AAQAOA_OK;
}

// ------------------------------------------------- pass plans, autotune
// A layer's qubits per pass (the low pass's qubit count L and the number K of
// high passes) for the forward (nv = 1) and the two-vector adjoint (nv = 2)
// passes. 0 selects the default of build_passes().
static int set_layers(aaqaoa_plan *pl, const int plan4[4])
{
    if (pl->small())
        return AAQAOA_OK;
    std::vector<Pass> v[2];
    for (int nv = 1; nv <= 2; nv++) {
        int T, CB, HB, L, K;
        pass_geometry(pl->c128, nv, &T, &CB, &HB);
        const int L2 = low_two_stage_bits(pl->c128, nv);
        default_layer(pl->n, T, CB, HB, L2, &L, &K, nv == 2);
        if (plan4[2 * (nv - 1)] > 0)
            L = plan4[2 * (nv - 1)];
        if (plan4[2 * (nv - 1) + 1] > 0)
            K = plan4[2 * (nv - 1) + 1];
        if (!layer_passes(pl->n, T, CB, HB, L2, L, K, v[nv - 1], nv == 2 && !pl->c128, nv == 2))
            return fail(AAQAOA_ERR_INVALID_ARG, "%s plan: low pass of %d qubits + %d high passes does not tile n=%d",
                        nv == 1 ? "forward" : "adjoint", L, K, pl->n);
    }
    pl->passes = v[0];
    pl->bwd_passes = v[1];
    pl->state_valid = false;
    return build_maps(pl);
}

int aaqaoa_get_pass_plan(aaqaoa_plan *pl, int *plan4)
{
    if (!pl || !plan4)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan or plan4 is NULL");
    plan4[0] = pl->passes.empty() ? 0 : pl->passes[0].qubits;
    plan4[1] = pl->passes.empty() ? 0 : (int)pl->passes.size() - 1;
    plan4[2] = pl->bwd_passes.empty() ? 0 : pl->bwd_passes[0].qubits;
    plan4[3] = pl->bwd_passes.empty() ? 0 : (int)pl->bwd_passes.size() - 1;
    return AAQAOA_OK;
}

int aaqaoa_set_pass_plan(aaqaoa_plan *pl, int fwd_low, int fwd_high, int bwd_low, int bwd_high)
{
    g_detail.clear();
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    if (fwd_low < 0 || fwd_high < 0 || bwd_low < 0 || bwd_high < 0)
        return fail(AAQAOA_ERR_INVALID_ARG, "negative pass-plan entry");
    const int plan4[4] = {fwd_low, fwd_high, bwd_low, bwd_high};
    return set_layers(pl, plan4);
}

int aaqaoa_set_layer_fusion(aaqaoa_plan *pl, int enable)
{
    g_detail.clear();
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    if (enable != 0 && enable != 1)
        return fail(AAQAOA_ERR_INVALID_ARG, "enable must be 0 or 1 (got %d)", enable);
    pl->fuse = enable != 0;
    pl->state_valid = false;
    return AAQAOA_OK;
}

int aaqaoa_get_layer_fusion(aaqaoa_plan *pl, int *enable)
{
    if (!pl || !enable)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan or enable is NULL");
    *enable = pl->fuse ? 1 : 0;
    return AAQAOA_OK;
}

int aaqaoa_get_schedule(aaqaoa_plan *pl, int adjoint, int32_t *steps, int cap, int *count)
{
    if (!pl || !count || cap < 0 || (cap > 0 && !steps) || adjoint < 0 || adjoint > 2)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan/count is NULL, cap < 0, steps is NULL or adjoint not 0/1/2");
    const bool bwd = adjoint == 1;
    const std::vector<Pass> &passes = bwd ? pl->bwd_passes : pl->passes;
    const Turn tn = adjoint ? turnaround(pl) : Turn{};  // gradient evaluations only
    std::vector<Step> sched = bwd ? layer_schedule(pl->p, passes, plan_fuses(pl), true, false, -1, tn.kb)
                                  : layer_schedule(pl->p, passes, plan_fuses(pl), false, !pl->c128, tn.kf);
    if (adjoint == 2 && tn.kf >= 0)
        sched.pop_back();  // the turnaround applies the forward's last group
    if (bwd && tn.kb >= 0)  // the turnaround first: the last layer on its group, forward then back
        sched.insert(sched.begin(), Step{tn.kb, pl->p - 1, pl->p - 1, 0, true, false});
    *count = (int)sched.size();
    for (int i = 0; i < cap && i < (int)sched.size(); i++) {
        const Pass &ps = passes[sched[i].k];
        steps[5 * i + 0] = ps.is_low ? 0 : ps.s;
        steps[5 * i + 1] = ps.qubits;
        steps[5 * i + 2] = sched[i].layer;
        steps[5 * i + 3] = sched[i].layer2;
        steps[5 * i + 4] = sched[i].j0;
    }
    return AAQAOA_OK;
}

namespace {
struct TuneKey {
    int dev, c128, n, p, cap, grad, fuse;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(dev, c128, n, p, cap, grad, fuse) < std::tie(o.dev, o.c128, o.n, o.p, o.cap, o.grad, o.fuse);
    }
};
std::map<TuneKey, std::array<int, 4>> &plan_tune_cache()
{
    static std::map<TuneKey, std::array<int, 4>> cache;
    return cache;
}

// candidate (L, K) of one pass kind: the fewest and one more high pass, each
// with the full low pass and with the two-stage one
std::vector<std::array<int, 2>> layer_candidates(const aaqaoa_plan *pl, int nv)
{
    int T, CB, HB, L, K;
    pass_geometry(pl->c128, nv, &T, &CB, &HB);
    const int L2 = low_two_stage_bits(pl->c128, nv);
    default_layer(pl->n, T, CB, HB, L2, &L, &K, nv == 2);
    std::vector<std::array<int, 2>> c;
    const bool cl = nv == 2 && !pl->c128;
    for (int k = (cl && K > 1 ? K - 1 : K); k <= K + 1; k++)
        for (int l : {T, L2, CLUSTER_LOW_QUBITS}) {
            std::vector<Pass> v;
            if (layer_passes(pl->n, T, CB, HB, L2, l, k, v, cl, nv == 2) &&
                std::find(c.begin(), c.end(), std::array<int, 2>{l, k}) == c.end())
                c.push_back({l, k});
        }
    return c;
}

float time_ms(cudaStream_t st, const std::function<int()> &work, int reps)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
    int r = 0;
    for (int i = 0; i < reps && !r; i++)
        r = work();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return r ? 1e30f : ms / reps;
}
}  // namespace

int aaqaoa_autotune(aaqaoa_plan *pl, int *plan4)
{
    g_detail.clear();
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    if (!pl->ws)
        return fail(AAQAOA_ERR_WORKSPACE, "no workspace set (aaqaoa_set_workspace)");
    int r = AAQAOA_OK;
    const char *env = std::getenv("AAQAOA_AUTOTUNE");
    if (!pl->small() && !(env && env[0] == '0')) {
        int dev = 0;
        cudaGetDevice(&dev);
        const TuneKey key{dev, pl->c128 ? 1 : 0, pl->n, pl->p, pl->cap, pl->ws_grad ? 1 : 0, plan_fuses(pl) ? 1 : 0};
        auto it = plan_tune_cache().find(key);
        if (it != plan_tune_cache().end()) {
            r = set_layers(pl, it->second.data());
        } else {
            std::vector<double> g(pl->p), b(pl->p);
            for (int l = 0; l < pl->p; l++) {
                g[l] = 0.3 + 0.1 * l;
                b[l] = 0.2 + 0.05 * l;
            }
            if ((r = upload_params(pl, 1, g.data(), b.data())) ||
                (r = enqueue_params(pl, 1, pl->d_params(), pl->d_params() + pl->p)))
                return r;
            const FwdMode fm = pl->ws_grad ? FWD_GRAD : FWD_ENERGY;
            std::array<int, 4> best{0, 0, 0, 0};
            float best_ms = 1e30f;
            for (auto &c : layer_candidates(pl, 1)) {
                const int cand[4] = {c[0], c[1], 0, 0};
                if ((r = set_layers(pl, cand)))
                    return r;
                auto run = [&]() { return enqueue_forward(pl, 1, AAQAOA_OBS_FULL, fm); };
                time_ms(pl->stream, run, 1);
                const float ms = time_ms(pl->stream, run, 2);
                if (ms < best_ms) {
                    best_ms = ms;
                    best[0] = c[0];
                    best[1] = c[1];
                }
            }
            if (pl->ws_grad) {
                best_ms = 1e30f;
                for (auto &c : layer_candidates(pl, 2)) {
                    const int cand[4] = {best[0], best[1], c[0], c[1]};
                    if ((r = set_layers(pl, cand)))
                        return r;
                    if ((r = enqueue_forward(pl, 1, AAQAOA_OBS_FULL, FWD_GRAD)))
                        return r;
                    auto run = [&]() { return enqueue_backward(pl, 1, AAQAOA_OBS_FULL); };
                    time_ms(pl->stream, run, 1);
                    const float ms = time_ms(pl->stream, run, 2);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best[2] = c[0];
                        best[3] = c[1];
                    }
                }
            }
            if ((r = set_layers(pl, best.data())))
                return r;
            std::vector<double> rows;
            if ((r = fetch_out(pl, 1, rows)))  // a device timeout during tuning surfaces here
                return r;
            plan_tune_cache()[key] = best;
        }
    }
    if (!r && plan4)
        r = aaqaoa_get_pass_plan(pl, plan4);
    return r;
}

int aaqaoa_set_stream(aaqaoa_plan *pl, void *stream)
{
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    pl->stream = (cudaStream_t)stream;
    return AAQAOA_OK;
}

int aaqaoa_expect(aaqaoa_plan *pl, const double *gamma, const double *beta, int observable, int agg_mode,
                  double *energy)
{
    g_detail.clear();
    int r = check_ready(pl, observable, false, 1);
    if (r)
        return r;
    if (agg_mode < AAQAOA_AGG_FUSED || agg_mode > AAQAOA_AGG_SINGLEPASS)
        return fail(AAQAOA_ERR_INVALID_ARG, "agg_mode %d unknown", agg_mode);
    if (pl->ising && agg_mode != AAQAOA_AGG_FUSED)
        return fail(AAQAOA_ERR_UNSUPPORTED, "Ising plans aggregate in the fused mode only");
    if (!energy)
        return fail(AAQAOA_ERR_INVALID_ARG, "energy is NULL");
    pl->launches = 0;
    if ((r = upload_params(pl, 1, gamma, beta)))
        return r;
    if ((r = enqueue_expect(pl, 1, pl->d_params(), pl->d_params() + pl->p, observable, agg_mode)))
        return r;
    std::vector<double> rows;
    if ((r = fetch_out(pl, 1, rows)))
        return r;
    *energy = rows[0];
    return AAQAOA_OK;
}

int aaqaoa_grad(aaqaoa_plan *pl, const double *gamma, const double *beta, int observable, double *energy,
                double *dgamma, double *dbeta)
{
    g_detail.clear();
    int r = check_ready(pl, observable, true, 1);
    if (r)
        return r;
    if (!energy || !dgamma || !dbeta)
        return fail(AAQAOA_ERR_INVALID_ARG, "output pointer is NULL");
    pl->launches = 0;
    if ((r = upload_params(pl, 1, gamma, beta)))
        return r;
    if ((r = enqueue_grad(pl, pl->d_params(), pl->d_params() + pl->p, observable)))
        return r;
    std::vector<double> rows;
    if ((r = fetch_out(pl, 1, rows)))
        return r;
    *energy = rows[0];
    for (int l = 0; l < pl->p; l++) {
        dgamma[l] = rows[1 + l];
        dbeta[l] = rows[1 + pl->p + l];
    }
    return AAQAOA_OK;
}

int aaqaoa_expect_batch(aaqaoa_plan *pl, int B, const double *gamma, const double *beta, int observable,
                        double *energy)
{
    g_detail.clear();
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    if (B < 1 || !energy)
        return fail(AAQAOA_ERR_INVALID_ARG, "B < 1 or energy NULL");
    int r = check_ready(pl, observable, false, 1);
    if (r)
        return r;
    pl->launches = 0;
    std::vector<double> rows;
    for (int b0 = 0; b0 < B; b0 += pl->cap) {
        const int Bw = B - b0 < pl->cap ? B - b0 : pl->cap;
        if ((r = upload_params(pl, Bw, gamma + (size_t)b0 * pl->p, beta + (size_t)b0 * pl->p)))
            return r;
        if ((r = enqueue_expect(pl, Bw, pl->d_params(), pl->d_params() + (size_t)Bw * pl->p, observable,
                                AAQAOA_AGG_FUSED)))
            return r;
        if ((r = fetch_out(pl, Bw, rows)))
            return r;
        for (int b = 0; b < Bw; b++)
            energy[b0 + b] = rows[(size_t)b * pl->out_stride()];
    }
    return AAQAOA_OK;
}

int aaqaoa_grad_batch(aaqaoa_plan *pl, int B, const double *gamma, const double *beta, int observable,
                      double *energy, double *dgamma, double *dbeta)
{
    g_detail.clear();
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    if (B < 1 || !energy || !dgamma || !dbeta)
        return fail(AAQAOA_ERR_INVALID_ARG, "B < 1 or an output pointer is NULL");
    int r = check_ready(pl, observable, true, 1);
    if (r)
        return r;
    pl->launches = 0;
    const int p = pl->p;
    std::vector<double> rows;
    for (int b0 = 0; b0 < B; b0 += pl->cap) {  // waves of at most the workspace's batch size
        const int Bw = B - b0 < pl->cap ? B - b0 : pl->cap;
        if ((r = upload_params(pl, Bw, gamma + (size_t)b0 * p, beta + (size_t)b0 * p)))
            return r;
        if ((r = enqueue_grad(pl, pl->d_params(), pl->d_params() + (size_t)Bw * p, observable, Bw)))
            return r;
        if ((r = fetch_out(pl, Bw, rows)))
            return r;
        for (int b = 0; b < Bw; b++) {
            const double *row = &rows[(size_t)b * pl->out_stride()];
            energy[b0 + b] = row[0];
            for (int l = 0; l < p; l++) {
                dgamma[(size_t)(b0 + b) * p + l] = row[1 + l];
                dbeta[(size_t)(b0 + b) * p + l] = row[1 + p + l];
            }
        }
    }
    return AAQAOA_OK;
}

int aaqaoa_grad_batch_device(aaqaoa_plan *pl, int B, const double *d_gamma, const double *d_beta, int observable,
                             double *d_out)
{
    g_detail.clear();
    int r = check_ready(pl, observable, true, B);
    if (r)
        return r;
    if (!d_gamma || !d_beta || !d_out)
        return fail(AAQAOA_ERR_INVALID_ARG, "device pointer is NULL");
    pl->launches = 0;
    if ((r = enqueue_grad(pl, d_gamma, d_beta, observable, B)))
        return r;
    CK(cudaMemcpyAsync(d_out, pl->d_out(), (size_t)B * pl->out_stride() * sizeof(double), cudaMemcpyDeviceToDevice,
                       pl->stream));
    return AAQAOA_OK;
}

int aaqaoa_expect_device(aaqaoa_plan *pl, int B, const double *d_gamma, const double *d_beta, int observable,
                         double *d_energy)
{
    g_detail.clear();
    int r = check_ready(pl, observable, false, B);
    if (r)
        return r;
    if (!d_gamma || !d_beta || !d_energy)
        return fail(AAQAOA_ERR_INVALID_ARG, "device pointer is NULL");
    pl->launches = 0;
    if ((r = enqueue_expect(pl, B, d_gamma, d_beta, observable, AAQAOA_AGG_FUSED)))
        return r;
    CK(cudaMemcpy2DAsync(d_energy, sizeof(double), pl->d_out(), pl->out_stride() * sizeof(double), sizeof(double),
                         B, cudaMemcpyDeviceToDevice, pl->stream));
    return AAQAOA_OK;
}

int aaqaoa_grad_device(aaqaoa_plan *pl, const double *d_gamma, const double *d_beta, int observable, double *d_out)
{
    g_detail.clear();
    int r = check_ready(pl, observable, true, 1);
    if (r)
        return r;
    if (!d_gamma || !d_beta || !d_out)
        return fail(AAQAOA_ERR_INVALID_ARG, "device pointer is NULL");
    pl->launches = 0;
    if ((r = enqueue_grad(pl, d_gamma, d_beta, observable)))
        return r;
    CK(cudaMemcpyAsync(d_out, pl->d_out(), pl->out_stride() * sizeof(double), cudaMemcpyDeviceToDevice, pl->stream));
    return AAQAOA_OK;
}

int aaqaoa_sync(aaqaoa_plan *pl)
{
    if (!pl || !pl->ws)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan NULL or without workspace");
    std::vector<double> rows;
    return fetch_out(pl, 1, rows);
}

int aaqaoa_statevector(aaqaoa_plan *pl, const double *gamma, const double *beta, void *host_out)
{
    g_detail.clear();
    int r = check_ready(pl, AAQAOA_OBS_FULL, false, 1);
    if (r)
        return r;
    if (!host_out)
        return fail(AAQAOA_ERR_INVALID_ARG, "host_out is NULL");
    pl->launches = 0;
    if ((r = upload_params(pl, 1, gamma, beta)))
        return r;
    if ((r = enqueue_params(pl, 1, pl->d_params(), pl->d_params() + pl->p)))
        return r;
    if (pl->small()) {
        SmallArgs s = small_args(pl, AAQAOA_OBS_FULL, SMALL_ENERGY, 1);
        CKL(launch_small(pl->c128, s, 1, pl->stream), "whole-circuit kernel");
        pl->launches++;
    } else {
        if ((r = enqueue_forward(pl, 1, AAQAOA_OBS_FULL, FWD_STATE)))
            return r;
        // the passes store the twisted, shifted-angle state: map it back
        CKL(launch_untwist(pl->c128, pl->d_phi(), pl->n, pl->d_cs(), pl->p, pl->ising ? 1 : 0, pl->stream),
            "statevector export");
        pl->launches++;
    }
    pl->state_valid = true;
    std::vector<double> rows;
    if ((r = fetch_out(pl, 1, rows)))
        return r;
    CK(cudaMemcpy(host_out, pl->d_phi(), ((size_t)1 << pl->n) * pl->amp(), cudaMemcpyDeviceToHost));
    return AAQAOA_OK;
}

int aaqaoa_edge_zz(aaqaoa_plan *pl, const double *gamma, const double *beta, double *zz)
{
    g_detail.clear();
    int r = check_ready(pl, AAQAOA_OBS_FULL, false, 1);
    if (r)
        return r;
    if (!zz)
        return fail(AAQAOA_ERR_INVALID_ARG, "zz is NULL");
    pl->launches = 0;
    if ((r = upload_params(pl, 1, gamma, beta)))
        return r;
    if ((r = enqueue_params(pl, 1, pl->d_params(), pl->d_params() + pl->p)))
        return r;
    if (pl->small()) {
        SmallArgs s = small_args(pl, AAQAOA_OBS_FULL, SMALL_ENERGY, 1);
        CKL(launch_small(pl->c128, s, 1, pl->stream), "whole-circuit kernel");
        pl->launches++;
    } else if ((r = enqueue_forward(pl, 1, AAQAOA_OBS_FULL, FWD_STATE))) {
        return r;
    }
    pl->state_valid = true;
    const int grid = pl->n < 10 ? 1 : agg_grid(pl->c128);
    for (int t0 = 0; t0 < pl->m; t0 += 64) {
        AggArgs a;
        memset(&a, 0, sizeof a);
        a.n = pl->n;
        a.chunks = pl->n < 10 ? 0 : ((uint64_t)1 << (pl->n - 10));
        a.state = pl->d_phi();
        a.partials = pl->d_partials();
        a.counter = pl->d_counter_agg();
        a.out_terms = pl->d_zz() + t0;
        a.out_energy = pl->d_out();
        a.num_terms = pl->m - t0 < 64 ? pl->m - t0 : 64;
        for (int t = 0; t < a.num_terms; t++) {
            a.term_u[t] = pl->edges[2 * (t0 + t)];
            a.term_v[t] = pl->edges[2 * (t0 + t) + 1];
            a.term_w[t] = 1.0;
        }
        CKL(launch_agg_terms(pl->c128, a, pl->stream, grid), "edge <ZZ> pass");
        pl->launches++;
    }
    std::vector<double> rows;
    if ((r = fetch_out(pl, 1, rows)))
        return r;
    if (pl->m > 0)
        CK(cudaMemcpy(zz, pl->d_zz(), pl->m * sizeof(double), cudaMemcpyDeviceToHost));
    return AAQAOA_OK;
}

int aaqaoa_verify_orbits(aaqaoa_plan *pl, const double *gamma, const double *beta, double tol, int *bad_orbit)
{
    g_detail.clear();
    if (!pl || !bad_orbit)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan or bad_orbit is NULL");
    *bad_orbit = -1;
    if (pl->num_orbits == 0 || pl->edge_orbit.empty())
        return fail(AAQAOA_ERR_INVALID_ARG, "the plan was prepared without edge_orbit: class membership unknown");
    if (!(tol >= 0.0))
        return fail(AAQAOA_ERR_INVALID_ARG, "tolerance %g is not >= 0", tol);
    std::vector<double> zz((size_t)pl->m);
    int r = aaqaoa_edge_zz(pl, gamma, beta, zz.data());
    if (r)
        return r;
    for (int e = 0; e < pl->m; e++) {
        const int c = pl->edge_orbit[e], rep = pl->orbit_rep[c];
        const double d = std::fabs(zz[e] - zz[rep]);
        if (d > tol) {
            *bad_orbit = c;
            return fail(AAQAOA_ERR_BAD_ORBITS, "edge %d differs from the representative %d of orbit %d by %.3g in <ZZ>",
                        e, rep, c, d);
        }
    }
    return AAQAOA_OK;
}

int aaqaoa_max_cut(aaqaoa_plan *pl, int32_t *c_max, uint64_t *argmax)
{
    g_detail.clear();
    if (!pl || !c_max || !argmax)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan, c_max or argmax is NULL");
    if (!pl->ws)
        return fail(AAQAOA_ERR_WORKSPACE, "no workspace set (aaqaoa_set_workspace)");
    if (pl->ising)
        return fail(AAQAOA_ERR_UNSUPPORTED, "the maximum cut needs an integer cut function (not an Ising plan)");
    (void)cudaGetLastError();
    CK(cudaMemsetAsync(pl->d_maxcut_key(), 0, sizeof(unsigned long long), pl->stream));
    CKL(launch_maxcut(pl->cost, pl->n, pl->d_maxcut_key(), pl->stream), "maximum cut");
    unsigned long long key = 0;
    CK(cudaMemcpyAsync(&key, pl->d_maxcut_key(), sizeof key, cudaMemcpyDeviceToHost, pl->stream));
    CK(cudaStreamSynchronize(pl->stream));
    const unsigned long long low = (1ull << 35) - 1ull;
    *c_max = (int32_t)(key >> 35);
    *argmax = (uint64_t)(low - (key & low));
    return AAQAOA_OK;
}

int aaqaoa_sample(aaqaoa_plan *pl, const double *gamma, const double *beta, int K, const double *u,
                  uint64_t *x_out, int32_t *cut_out)
{
    g_detail.clear();
    int r = check_ready(pl, AAQAOA_OBS_FULL, false, 1);
    if (r)
        return r;
    if (K < 1 || K > AAQAOA_SAMPLE_MAX)
        return fail(AAQAOA_ERR_INVALID_ARG, "K = %d outside [1, %d]", K, AAQAOA_SAMPLE_MAX);
    if (pl->ising)
        return fail(AAQAOA_ERR_UNSUPPORTED, "sampling reports integer cut values (not an Ising plan)");
    if (!u || !x_out)
        return fail(AAQAOA_ERR_INVALID_ARG, "u or x_out is NULL");
    for (int k = 0; k < K; k++)
        if (!(u[k] >= 0.0 && u[k] < 1.0))
            return fail(AAQAOA_ERR_INVALID_ARG, "u[%d] = %g is not in [0, 1)", k, u[k]);
    pl->launches = 0;
    if ((r = upload_params(pl, 1, gamma, beta)))
        return r;
    if ((r = enqueue_params(pl, 1, pl->d_params(), pl->d_params() + pl->p)))
        return r;
    if (pl->small()) {
        SmallArgs s = small_args(pl, AAQAOA_OBS_FULL, SMALL_ENERGY, 1);
        CKL(launch_small(pl->c128, s, 1, pl->stream), "whole-circuit kernel");
        pl->launches++;
    } else if ((r = enqueue_forward(pl, 1, AAQAOA_OBS_FULL, FWD_STATE))) {
        return r;
    }
    pl->state_valid = true;
    CK(cudaMemcpyAsync(pl->d_samp_u(), u, (size_t)K * sizeof(double), cudaMemcpyHostToDevice, pl->stream));
    CKL(launch_sample(pl->c128, pl->d_phi(), pl->n, pl->d_samp_sums(), pl->d_samp_total(), K, pl->d_samp_u(),
                      pl->d_samp_x(), cut_out ? pl->d_samp_cut() : nullptr, pl->cost, pl->stream),
        "sampling");
    pl->launches += 3;
    std::vector<double> rows;
    if ((r = fetch_out(pl, 1, rows)))
        return r;
    CK(cudaMemcpy(x_out, pl->d_samp_x(), (size_t)K * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (cut_out)
        CK(cudaMemcpy(cut_out, pl->d_samp_cut(), (size_t)K * sizeof(int32_t), cudaMemcpyDeviceToHost));
    return AAQAOA_OK;
}

int aaqaoa_aggregate_only(aaqaoa_plan *pl, int observable, int agg_mode, double *energy)
{
    g_detail.clear();
    int r = check_ready(pl, observable, false, 1);
    if (r)
        return r;
    if (!energy)
        return fail(AAQAOA_ERR_INVALID_ARG, "energy is NULL");
    if (agg_mode != AAQAOA_AGG_PERTERM && agg_mode != AAQAOA_AGG_SINGLEPASS)
        return fail(AAQAOA_ERR_INVALID_ARG, "aggregate_only needs PERTERM or SINGLEPASS");
    if (pl->ising)
        return fail(AAQAOA_ERR_UNSUPPORTED, "Ising plans aggregate in the fused mode only");
    if (!pl->state_valid)
        return fail(AAQAOA_ERR_INVALID_ARG, "no stored state: run aaqaoa_statevector or a non-fused expect first");
    pl->launches = 0;
    if ((r = enqueue_aggregate(pl, observable, agg_mode)))
        return r;
    std::vector<double> rows;
    if ((r = fetch_out(pl, 1, rows)))
        return r;
    *energy = rows[0];
    return AAQAOA_OK;
}

int aaqaoa_inject_fault(aaqaoa_plan *pl, int kind)
{
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    if (kind != 0 && kind != AAQAOA_FAULT_DROP_TILE)
        return fail(AAQAOA_ERR_INVALID_ARG, "fault kind %d unknown", kind);
    if (kind == AAQAOA_FAULT_DROP_TILE && pl->small())
        return fail(AAQAOA_ERR_UNSUPPORTED, "n=%d runs in one CTA: no tiled pass to drop a tile from", pl->n);
    pl->inject = kind;
    return AAQAOA_OK;
}

int aaqaoa_plan_info(const aaqaoa_plan *pl, int *n, int *p, int *num_edges, int *num_orbits, unsigned *flags)
{
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    if (n) *n = pl->n;
    if (p) *p = pl->p;
    if (num_edges) *num_edges = pl->m;
    if (num_orbits) *num_orbits = pl->num_orbits;
    if (flags) *flags = pl->c128 ? AAQAOA_C128 : AAQAOA_C64;
    return AAQAOA_OK;
}

int aaqaoa_launch_count(const aaqaoa_plan *pl, int *launches)
{
    if (!pl || !launches)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan or launches NULL");
    *launches = pl->launches;
    return AAQAOA_OK;
}

int aaqaoa_profile_enable(aaqaoa_plan *pl, int enable)
{
    if (!pl)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan is NULL");
    for (auto &r : pl->prof_recs) {
        pl->prof_pool.push_back(r.a);
        pl->prof_pool.push_back(r.b);
    }
    pl->prof_recs.clear();
    pl->prof = enable != 0;
    return AAQAOA_OK;
}

int aaqaoa_profile_read(aaqaoa_plan *pl, int kind, double *ms_total, int *launches, double *bytes)
{
    if (!pl || kind < 0 || kind >= PK_COUNT)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan NULL or kind %d unknown", kind);
    CK(cudaStreamSynchronize(pl->stream));
    double ms = 0.0, by = 0.0;
    int cnt = 0;
    for (auto &r : pl->prof_recs) {
        if (r.kind != kind)
            continue;
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        ms += t;
        by += r.bytes;
        cnt++;
    }
    if (ms_total) *ms_total = ms;
    if (launches) *launches = cnt;
    if (bytes) *bytes = by;
    return AAQAOA_OK;
}

int aaqaoa_stats(aaqaoa_plan *pl, aaqaoa_stats_t *out)
{
    if (!pl || !out)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan or out is NULL");
    static_assert(AAQAOA_STAT_KINDS == PK_COUNT, "one stats entry per kernel kind");
    for (int k = 0; k < PK_COUNT; k++) {
        int r = aaqaoa_profile_read(pl, k, &out->ms[k], &out->launches[k], &out->bytes[k]);
        if (r)
            return r;
    }
    return AAQAOA_OK;
}

int aaqaoa_profile_launches(aaqaoa_plan *pl, int max, int *count, int *kind, int *flags, double *ms, double *bytes)
{
    if (!pl || !count || max < 0)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan or count NULL, or max < 0");
    CK(cudaStreamSynchronize(pl->stream));
    *count = (int)pl->prof_recs.size();
    for (int i = 0; i < max && i < (int)pl->prof_recs.size(); i++) {
        const auto &r = pl->prof_recs[i];
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        if (kind) kind[i] = r.kind;
        if (flags) flags[i] = r.flags;
        if (ms) ms[i] = t;
        if (bytes) bytes[i] = r.bytes;
    }
    return AAQAOA_OK;
}

void aaqaoa_destroy(aaqaoa_plan *pl)
{
    if (!pl)
        return;
    for (auto &r : pl->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : pl->prof_pool)
        cudaEventDestroy(e);
    delete pl;
}

}  // extern "C"

// ====================================================== static scratch
// An energy evaluation for callers that cannot allocate device memory. All of
// its device scratch (control words, phase tables, parameters, partial sums
// and one statevector) lives in this file-scope array, which every GPU that
// loads the library holds until the process exits.
namespace {

constexpr size_t STATIC_FIXED_BYTES = (size_t)1 << 20;   // control, outputs, tables, partials
constexpr size_t STATIC_STATE_BYTES = (size_t)32 << 20;  // one statevector
constexpr size_t STATIC_SCRATCH_BYTES = STATIC_FIXED_BYTES + STATIC_STATE_BYTES;
constexpr int STATIC_MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

std::mutex g_static_mutex;
unsigned char *g_static_ptr[STATIC_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side name of a __device__ array is not a device
// address).
int static_scratch(unsigned char **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= STATIC_MAX_DEVICES)
        return fail(AAQAOA_ERR_UNSUPPORTED, "device ordinal %d beyond the static scratch table", dev);
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_ptr[dev];
    return AAQAOA_OK;
}

}  // namespace

extern "C" int aaqaoa_expect_static(aaqaoa_plan *pl, const double *gamma, const double *beta, int observable,
                                    double *energy)
{
    g_detail.clear();
    if (!pl || !gamma || !beta || !energy)
        return fail(AAQAOA_ERR_INVALID_ARG, "plan, gamma, beta or energy is NULL");
    if (observable != AAQAOA_OBS_FULL && observable != AAQAOA_OBS_RED)
        return fail(AAQAOA_ERR_INVALID_ARG, "observable %d unknown", observable);
    if (observable == AAQAOA_OBS_RED && pl->num_orbits == 0)
        return fail(AAQAOA_ERR_INVALID_ARG, "H_red requested but the plan has no edge orbits");
    if (pl->ising)
        return fail(AAQAOA_ERR_UNSUPPORTED, "the static-scratch entry point takes MaxCut plans only");
    const size_t state_bytes = ((size_t)1 << pl->n) * pl->amp();
    if (state_bytes > STATIC_STATE_BYTES)
        return fail(AAQAOA_ERR_UNSUPPORTED,
                    "static scratch holds one statevector of at most %zu bytes (n <= %d for %s); n = %d needs %zu",
                    STATIC_STATE_BYTES, pl->c128 ? 21 : 22, pl->c128 ? "complex128" : "complex64", pl->n,
                    state_bytes);
    unsigned char *base = nullptr;
    int r = static_scratch(&base);
    if (r)
        return r;

    // fixed region: [ctrl 256 | out | gamma, beta | cs | tables | partials]
    const int p = pl->p;
    size_t off = 256;
    double *d_out = reinterpret_cast<double *>(base + off);
    off = align256(off + (size_t)pl->out_stride() * sizeof(double));
    double *d_par = reinterpret_cast<double *>(base + off);
    off = align256(off + 2 * (size_t)p * sizeof(double));
    double2 *d_cs = reinterpret_cast<double2 *>(base + off);
    off = align256(off + (size_t)p * sizeof(double2));
    void *d_tab = base + off;  // exact, forward-scaled and inverse tables
    off = align256(off + 3 * (size_t)p * pl->tab_len() * pl->amp());
    double *d_part = reinterpret_cast<double *>(base + off);
    off = align256(off + 3 * (size_t)device_sms() * sizeof(double));
    if (off > STATIC_FIXED_BYTES)
        return fail(AAQAOA_ERR_UNSUPPORTED, "tables for p = %d and |E| = %d exceed the static scratch", p, pl->m);
    int *d_err = reinterpret_cast<int *>(base);
    unsigned *d_counter = reinterpret_cast<unsigned *>(base + 8);
    void *d_phi = base + STATIC_FIXED_BYTES;

    cudaStream_t st = pl->stream;
    (void)cudaGetLastError();
    // what must start at zero: error flag, last-block counters, the output row
    CK(cudaMemsetAsync(base, 0, 256, st));
    CK(cudaMemsetAsync(d_out, 0, (size_t)pl->out_stride() * sizeof(double), st));
    CK(cudaMemcpyAsync(d_par, gamma, (size_t)p * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(d_par + p, beta, (size_t)p * sizeof(double), cudaMemcpyHostToDevice, st));
    CKL(launch_params(pl->c128, 1, p, pl->tab_len(), pl->n, d_par, d_par + p, d_tab, d_cs, st), "parameter tables");

    if (pl->small()) {
        SmallArgs s;
        memset(&s, 0, sizeof s);
        s.n = pl->n;
        s.p = p;
        s.tab_len = pl->tab_len();
        s.mode = SMALL_ENERGY;
        s.write_state = 0;
        s.amp0 = std::pow(2.0, -0.5 * pl->n);
        s.tab = d_tab;
        s.cs = d_cs;
        s.out = d_out;
        s.out_stride = pl->out_stride();
        s.state = d_phi;
        s.obs = pl->obs[observable];
        s.cost = pl->cost;
        CKL(launch_small(pl->c128, s, 1, st), "whole-circuit kernel");
    } else {
        const int np = (int)pl->passes.size();
        CUtensorMap maps[8];
        if (np > 8)
            return fail(AAQAOA_ERR_UNSUPPORTED, "%d passes per layer", np);
        int wide[8];
        for (int k = 0; k < np; k++)
            if ((r = make_map(&maps[k], d_phi, pl->n, pl->passes[k].s, pl->passes[k].cb, pl->T(), pl->CB(), pl->amp(),
                              1, &wide[k])))
                return r;
        const int grid = pass_grid(pl->tiles());
        const std::vector<Step> sched = layer_schedule(p, pl->passes, plan_fuses(pl), false, !pl->c128);
        for (size_t i = 0; i < sched.size(); i++) {
            const int k = sched[i].k;
            // the plan's own pass arguments, pointed at the static scratch
            PassArgs a = forward_args(pl, observable, 1, sched[i], i, sched.size(), FWD_ENERGY);
            a.wide_rows = wide[k];
            a.tab = tab_kind(pl, d_tab, 1, 1);
            a.cs = d_cs;
            a.partials = d_part;
            a.counter = d_counter;
            a.out = d_out;
            a.err = d_err;
            a.pt = nullptr;
            CKL(launch_pass(pl->c128, 1, maps[k], maps[k], a, grid, st), "forward pass");
        }
    }
    int err = 0;
    CK(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(energy, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err)
        return fail(AAQAOA_ERR_TIMEOUT, "a bounded device wait expired (TMA tile never arrived)");
    return AAQAOA_OK;
}

// ============================================== uneven multi-graph batches
// Graphs with n up to the tile size run together in one k_small_multi launch;
// larger graphs each own a tiled sub-plan. One evaluation of the batch is
// captured into a CUDA graph whose large-graph work is spread over `branches`
// parallel streams; the branch count is chosen by timing (autotune) on the
// first call for each observable and cached for the process.
struct aaqaoa_multi {
    int G = 0, p = 0;
    bool c128 = false;
    cudaStream_t stream = nullptr;  // the caller's stream: uploads, graph launch, downloads
    cudaStream_t cap = nullptr;     // private stream the evaluation is captured on
    std::vector<aaqaoa_plan *> plans;  // one per graph (validation + host tables)
    std::vector<int> small_idx, large_idx;
    // Graphs too large for one CTA run in groups of equal n: one batched pass
    // sequence per group, point b of the group being its b-th graph. Rows of
    // the parameter and energy arrays follow `order` (small graphs first,
    // then each group's members), so a group's rows are contiguous.
    struct Group {
        int n = 0, row0 = 0;
        std::vector<int> members;
        aaqaoa_plan *pl = nullptr;
        size_t off_fns = 0, off_ws = 0, ws_bytes = 0;
    };
    std::vector<Group> groups;
    std::vector<int> order;  // graph index of each row
    std::vector<SmallGraph> desc;       // small graphs, in small_idx order
    int small_max_n = 1, small_max_tab = 1;
    unsigned char *ws = nullptr;
    size_t ws_bytes = 0;
    size_t off_params = 0, off_energy = 0, off_desc = 0, off_err = 0;
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int branches[2] = {0, 0};
    int launches = 0;
};

namespace {

constexpr int MULTI_MAX_BRANCHES = 16;

size_t multi_layout(aaqaoa_multi *m)
{
    size_t off = 0;
    m->off_err = off;
    off += 256;
    m->off_params = off;
    off = align256(off + 2 * (size_t)m->G * m->p * sizeof(double));
    m->off_energy = off;
    off = align256(off + (size_t)m->G * sizeof(double));
    m->off_desc = off;
    off = align256(off + (m->desc.size() + 1) * sizeof(SmallGraph));
    for (auto &g : m->groups) {
        g.off_fns = off;
        off = align256(off + g.members.size() * sizeof(GraphFns));
        size_t b = 0;
        aaqaoa_workspace_bytes(g.pl, (int)g.members.size(), 0, &b);
        g.off_ws = off;
        g.ws_bytes = b;
        off = align256(off + b);
    }
    return off;
}

// everything one evaluation enqueues, on `origin` (+ side streams)
int multi_enqueue(aaqaoa_multi *m, int obs, int branches, cudaStream_t origin)
{
    if (branches > (int)m->side.size())
        branches = (int)m->side.size();
    double *d_par = reinterpret_cast<double *>(m->ws + m->off_params);
    double *d_en = reinterpret_cast<double *>(m->ws + m->off_energy);
    const size_t Gp = (size_t)m->G * m->p;
    m->launches = 0;
    CK(cudaEventRecord(m->fork, origin));
    for (int b = 0; b < branches; b++)
        CK(cudaStreamWaitEvent(m->side[b], m->fork, 0));
    if (!m->small_idx.empty()) {
        CKL(launch_small_multi(m->c128, reinterpret_cast<const SmallGraph *>(m->ws + m->off_desc),
                               (int)m->small_idx.size(), m->p, obs, m->small_max_n, m->small_max_tab, d_par,
                               d_par + Gp, d_en, origin),
            "small-graph batch kernel");
        m->launches++;
    }
    for (size_t j = 0; j < m->groups.size(); j++) {
        auto &g = m->groups[j];
        aaqaoa_plan *pl = g.pl;
        const int B = (int)g.members.size();
        cudaStream_t st = branches > 0 ? m->side[j % branches] : origin;
        pl->stream = st;
        pl->launches = 0;
        int r = enqueue_expect(pl, B, d_par + (size_t)g.row0 * m->p, d_par + Gp + (size_t)g.row0 * m->p, obs,
                               AAQAOA_AGG_FUSED);
        if (r)
            return r;
        m->launches += pl->launches;
        // energies: column 0 of the group's [B][1+2p] output rows
        CK(cudaMemcpy2DAsync(d_en + g.row0, sizeof(double), pl->d_out(), pl->out_stride() * sizeof(double),
                             sizeof(double), B, cudaMemcpyDeviceToDevice, st));
    }
    for (int b = 0; b < branches; b++) {
        CK(cudaEventRecord(m->join[b], m->side[b]));
        CK(cudaStreamWaitEvent(origin, m->join[b], 0));
    }
    return AAQAOA_OK;
}

int multi_capture(aaqaoa_multi *m, int obs, int branches, cudaGraphExec_t *exec)
{
    CK(cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal));
    int r = multi_enqueue(m, obs, branches, m->cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(m->cap, &graph);
    if (r) {
        if (graph)
            cudaGraphDestroy(graph);
        return r;
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGraphInstantiate");
    return AAQAOA_OK;
}

std::map<std::string, int> &autotune_cache()
{
    static std::map<std::string, int> c;
    return c;
}

std::string multi_signature(const aaqaoa_multi *m, int obs)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    std::string sig = "?";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess)
        sig = prop.name;
    char buf[64];
    snprintf(buf, sizeof buf, "|%d|%d|%d|", m->c128 ? 128 : 64, m->p, obs);
    sig += buf;
    for (auto &g : m->groups) {
        snprintf(buf, sizeof buf, "%dx%d,", g.n, (int)g.members.size());
        sig += buf;
    }
    return sig;
}

// choose the branch count by timing each candidate graph (3 launches each)
int multi_autotune(aaqaoa_multi *m, int obs)
{
    const int L = (int)m->groups.size();  // independent branches: one per group, at most one side stream each
    const std::string sig = multi_signature(m, obs);
    auto &cache = autotune_cache();
    const char *env = getenv("AAQAOA_AUTOTUNE");
    const bool tune = !(env && env[0] == '0');
    int best = L > 0 ? (L < 4 ? L : 4) : 0;
    if (cache.count(sig)) {
        best = cache[sig];
    } else if (tune && L > 1) {
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        float best_ms = 1e30f;
        for (int br = 1; br <= (int)m->side.size() && br <= L; br *= 2) {
            cudaGraphExec_t ex = nullptr;
            int r = multi_capture(m, obs, br, &ex);
            if (r) {
                cudaEventDestroy(a);
                cudaEventDestroy(b);
                return r;
            }
            cudaGraphLaunch(ex, m->stream);
            cudaEventRecord(a, m->stream);
            for (int i = 0; i < 3; i++)
                cudaGraphLaunch(ex, m->stream);
            cudaEventRecord(b, m->stream);
            cudaError_t e = cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            cudaGraphExecDestroy(ex);
            if (e != cudaSuccess) {
                cudaEventDestroy(a);
                cudaEventDestroy(b);
                return cuda_fail(e, "autotune run");
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = br;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cache[sig] = best;
    }
    m->branches[obs] = best;
    return multi_capture(m, obs, best, &m->exec[obs]);
}

}  // namespace

extern "C" {

int aaqaoa_prepare_multi(int G, const aaqaoa_graph_desc *graphs, int p, unsigned flags, void *stream,
                         aaqaoa_multi **out)
{
    g_detail.clear();
    if (!out)
        return fail(AAQAOA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (G < 1 || !graphs)
        return fail(AAQAOA_ERR_INVALID_ARG, "G=%d or graphs NULL", G);
    aaqaoa_multi *m = new (std::nothrow) aaqaoa_multi();
    if (!m)
        return fail(AAQAOA_ERR_INVALID_ARG, "out of host memory");
    m->G = G;
    m->p = p;
    m->c128 = flags == AAQAOA_C128;
    m->stream = (cudaStream_t)stream;
    for (int gi = 0; gi < G; gi++) {
        const aaqaoa_graph_desc &d = graphs[gi];
        aaqaoa_plan *pl = nullptr;
        int r = aaqaoa_prepare(d.n, d.num_edges, d.edges, d.num_orbits, d.orbit_rep, d.orbit_weight, d.edge_orbit, p,
                               flags, stream, &pl);
        if (r) {
            std::string why = g_detail;
            aaqaoa_destroy_multi(m);
            return fail(r, "graph %d: %s", gi, why.c_str());
        }
        m->plans.push_back(pl);
        if (pl->small()) {
            SmallGraph sg;
            memset(&sg, 0, sizeof sg);
            sg.gi = (int)m->small_idx.size();  // its row: small graphs come first
            sg.n = pl->n;
            sg.tab_len = pl->tab_len();
            for (int o = 0; o < 2; o++) {
                sg.K[o] = pl->obs[o].K;
                for (int k = 0; k < MAXK; k++) {
                    sg.w[o][k] = pl->obs[o].w[k];
                    for (int u = 0; u < MAXN; u++)
                        sg.obs[o][k][u] = pl->obs[o].nbr[k][u];
                }
            }
            for (int u = 0; u < MAXN; u++)
                sg.cost[u] = pl->cost.nbr[0][u];
            m->desc.push_back(sg);
            m->small_idx.push_back(gi);
            m->small_max_n = std::max(m->small_max_n, pl->n);
            m->small_max_tab = std::max(m->small_max_tab, pl->tab_len());
        } else {
            m->large_idx.push_back(gi);
        }
    }
    // rows: small graphs, then the large ones grouped by n (ascending)
    m->order = m->small_idx;
    std::map<int, std::vector<int>> by_n;
    for (int gi : m->large_idx)
        by_n[m->plans[gi]->n].push_back(gi);
    for (auto &kv : by_n) {
        aaqaoa_multi::Group g;
        g.n = kv.first;
        g.row0 = (int)m->order.size();
        g.members = kv.second;
        const aaqaoa_graph_desc &d = graphs[g.members[0]];
        int r = aaqaoa_prepare(d.n, d.num_edges, d.edges, d.num_orbits, d.orbit_rep, d.orbit_weight, d.edge_orbit, p,
                               flags, stream, &g.pl);
        if (r) {
            aaqaoa_destroy_multi(m);
            return r;
        }
        for (int gi : g.members)  // tables long enough for every member's cut values
            g.pl->wsum = std::max(g.pl->wsum, m->plans[gi]->wsum);
        m->order.insert(m->order.end(), g.members.begin(), g.members.end());
        m->groups.push_back(std::move(g));
    }
    const int nb = std::min<int>(MULTI_MAX_BRANCHES, std::max<int>(1, (int)m->groups.size()));
    for (int b = 0; b < nb; b++) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            aaqaoa_destroy_multi(m);
            return fail(AAQAOA_ERR_CUDA, "could not create the batch's side streams");
        }
        m->side.push_back(s);
        m->join.push_back(e);
    }
    if (cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess) {
        aaqaoa_destroy_multi(m);
        return fail(AAQAOA_ERR_CUDA, "could not create the batch's fork event");
    }
    *out = m;
    return AAQAOA_OK;
}

int aaqaoa_multi_workspace_bytes(const aaqaoa_multi *m, size_t *bytes)
{
    if (!m || !bytes)
        return fail(AAQAOA_ERR_INVALID_ARG, "multi or bytes NULL");
    *bytes = multi_layout(const_cast<aaqaoa_multi *>(m));
    return AAQAOA_OK;
}

int aaqaoa_multi_set_workspace(aaqaoa_multi *m, void *device_ptr, size_t bytes)
{
    if (!m)
        return fail(AAQAOA_ERR_INVALID_ARG, "multi is NULL");
    if (!device_ptr || ((uintptr_t)device_ptr & 255))
        return fail(AAQAOA_ERR_WORKSPACE, "workspace pointer NULL or not 256-byte aligned");
    const size_t need = multi_layout(m);
    if (bytes < need)
        return fail(AAQAOA_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", bytes, need);
    m->ws = (unsigned char *)device_ptr;
    m->ws_bytes = bytes;
    for (int o = 0; o < 2; o++)
        if (m->exec[o]) {
            cudaGraphExecDestroy(m->exec[o]);
            m->exec[o] = nullptr;
        }
    for (auto &g : m->groups) {
        int r = aaqaoa_set_workspace(g.pl, m->ws + g.off_ws, g.ws_bytes, (int)g.members.size(), 0);
        if (r)
            return r;
        g.pl->err_shared = reinterpret_cast<int *>(m->ws + m->off_err);
        std::vector<GraphFns> fns(g.members.size());
        for (size_t b = 0; b < g.members.size(); b++) {
            const aaqaoa_plan *q = m->plans[g.members[b]];
            fns[b].cost = q->cost;
            fns[b].obs[0] = q->obs[0];
            fns[b].obs[1] = q->obs[1];
        }
        CK(cudaMemcpyAsync(m->ws + g.off_fns, fns.data(), fns.size() * sizeof(GraphFns), cudaMemcpyHostToDevice,
                           m->stream));
        CK(cudaStreamSynchronize(m->stream));  // `fns` is a host temporary
        g.pl->pt_dev = reinterpret_cast<const GraphFns *>(m->ws + g.off_fns);
    }
    CK(cudaMemsetAsync(m->ws, 0, 256, m->stream));
    if (!m->desc.empty())
        CK(cudaMemcpyAsync(m->ws + m->off_desc, m->desc.data(), m->desc.size() * sizeof(SmallGraph),
                           cudaMemcpyHostToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
    return AAQAOA_OK;
}

int aaqaoa_expect_multi(aaqaoa_multi *m, const double *gamma, const double *beta, int observable, double *energy)
{
    g_detail.clear();
    if (!m || !gamma || !beta || !energy)
        return fail(AAQAOA_ERR_INVALID_ARG, "multi, gamma, beta or energy NULL");
    if (!m->ws)
        return fail(AAQAOA_ERR_WORKSPACE, "no workspace set (aaqaoa_multi_set_workspace)");
    if (observable != AAQAOA_OBS_FULL && observable != AAQAOA_OBS_RED)
        return fail(AAQAOA_ERR_INVALID_ARG, "observable %d unknown", observable);
    if (observable == AAQAOA_OBS_RED)
        for (int gi = 0; gi < m->G; gi++)
            if (m->plans[gi]->num_orbits == 0 && m->plans[gi]->m > 0)
                return fail(AAQAOA_ERR_INVALID_ARG, "H_red requested but graph %d has no edge orbits", gi);
    const size_t Gp = (size_t)m->G * m->p;
    double *d_par = reinterpret_cast<double *>(m->ws + m->off_params);
    std::vector<double> rows(2 * Gp), en((size_t)m->G);
    for (int r = 0; r < m->G; r++)
        for (int l = 0; l < m->p; l++) {
            rows[(size_t)r * m->p + l] = gamma[(size_t)m->order[r] * m->p + l];
            rows[Gp + (size_t)r * m->p + l] = beta[(size_t)m->order[r] * m->p + l];
        }
    CK(cudaMemcpyAsync(d_par, rows.data(), 2 * Gp * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    if (!m->exec[observable]) {
        // one direct run first (sets kernel attributes outside any capture)
        int r = multi_enqueue(m, observable, 0, m->stream);
        if (r)
            return r;
        CK(cudaStreamSynchronize(m->stream));
        if ((r = multi_autotune(m, observable)))
            return r;
    }
    CK(cudaGraphLaunch(m->exec[observable], m->stream));
    int err = 0;
    CK(cudaMemcpyAsync(&err, m->ws + m->off_err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CK(cudaMemcpyAsync(en.data(), m->ws + m->off_energy, (size_t)m->G * sizeof(double), cudaMemcpyDeviceToHost,
                       m->stream));
    CK(cudaStreamSynchronize(m->stream));
    for (int r = 0; r < m->G; r++)
        energy[m->order[r]] = en[r];
    if (err) {
        cudaMemsetAsync(m->ws, 0, 256, m->stream);
        cudaStreamSynchronize(m->stream);
        return fail(AAQAOA_ERR_TIMEOUT, "a bounded device wait expired in the batch");
    }
    return AAQAOA_OK;
}

int aaqaoa_multi_info(const aaqaoa_multi *m, int *G, int *small_graphs, int *branches, int *launches_per_call)
{
    if (!m)
        return fail(AAQAOA_ERR_INVALID_ARG, "multi is NULL");
    if (G) *G = m->G;
    if (small_graphs) *small_graphs = (int)m->small_idx.size();
    if (branches) *branches = std::max(m->branches[0], m->branches[1]);
    if (launches_per_call) *launches_per_call = m->launches;
    return AAQAOA_OK;
}

void aaqaoa_destroy_multi(aaqaoa_multi *m)
{
    if (!m)
        return;
    for (int o = 0; o < 2; o++)
        if (m->exec[o])
            cudaGraphExecDestroy(m->exec[o]);
    for (auto s : m->side)
        cudaStreamDestroy(s);
    for (auto e : m->join)
        cudaEventDestroy(e);
    if (m->fork)
        cudaEventDestroy(m->fork);
    if (m->cap)
        cudaStreamDestroy(m->cap);
    for (auto pl : m->plans)
        aaqaoa_destroy(pl);
    for (auto &g : m->groups)
        aaqaoa_destroy(g.pl);
    delete m;
}

}  // extern "C"

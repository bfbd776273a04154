// sm_103a kernels of the AA-QAOA hot path.
//
// The statevector is 2^n complex amplitudes (qubit i = bit i of the index).
// One QAOA layer (Eq. (1)) is a diagonal cost phase exp(-i gamma C(x)) followed
// by RX(2 beta) = exp(-i beta X) on every qubit (H_M = sum_i X_i). Both are
// HBM-streaming work, so the design is about moving every amplitude as few
// times as possible:
//
//  * A tile is 64 KB: 2^CB contiguous amplitudes (one 128-byte row) times 512
//    rows taken at stride 2^s along nine "high" qubits s..s+8. One TMA tensor
//    load (5-D box, 128-byte swizzle) stages it in shared memory; one TMA
//    store writes it back. A pass over all tiles applies the butterflies of up
//    to CB+9 qubits (low pass: qubits 0..CB+8 of a contiguous tile) or 9
//    qubits (high pass), so one layer takes ceil((n - CB - 9)/9) + 1 passes.
//  * Inside a tile the butterflies run in registers: each thread holds 2^RB
//    amplitudes that differ in RB chosen bits, applies the RB radix-2 stages,
//    and exchanges through (swizzled, bank-conflict-free) shared memory between
//    register stages.
//  * The cost phase of layer l is folded into the first register stage of the
//    layer's first pass; the reduction (energy), lambda = O psi, dE/dgamma and
//    the inverse cost phase are folded into the last stage of a pass. C(x) is
//    computed exactly in integers: per thread one cut value by popcount over
//    neighbour masks, then each of the thread's 2^RB amplitudes by flipping
//    register bits (cut change of a flipped vertex, corrected for flipped
//    neighbour pairs). The phase is a table lookup T_l[C(x)] of exp(-i gamma_l c)
//    built in FP64 with the argument reduced mod 2 pi.
//  * Reductions accumulate per thread in FP64 and are summed in a fixed order
//    by the last block of the grid, so results are bit-reproducible.
//
// Every wait on an mbarrier is bounded by a clock64 budget; on expiry the
// block sets the device error flag, waits once more (bounded) for its own TMA
// copies and returns without touching global memory.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "aaqaoa_internal.h"

namespace aaq {

// ---------------------------------------------------------------- helpers
template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

template <typename C, typename R>
__device__ __forceinline__ C mkc(R x, R y) { C r; r.x = x; r.y = y; return r; }

template <typename C>
__device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

template <typename C>
__device__ __forceinline__ C cmul_conj(C a, C b)  // a * conj(b)
{
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}

// (a, b) <- (c a - i s b, -i s a + c b): RX(2 beta) on one amplitude pair
template <typename C, typename R>
__device__ __forceinline__ void bfly(C &a, C &b, R c, R s)
{
    C a2, b2;
    a2.x = c * a.x + s * b.y;
    a2.y = c * a.y - s * b.x;
    b2.x = c * b.x + s * a.y;
    b2.y = c * b.y - s * a.x;
    a = a2;
    b = b2;
}

// Im(conj(l) f)
template <typename C>
__device__ __forceinline__ auto im_conj_mul(C l, C f) -> decltype(l.x) { return l.x * f.y - l.y * f.x; }

__host__ __device__ constexpr int hibit(int m) { return m >= 16 ? 4 : m >= 8 ? 3 : m >= 4 ? 2 : m >= 2 ? 1 : 0; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// ~1 s at 2 GHz
constexpr long long WAIT_BUDGET_CYCLES = 1ll << 31;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > WAIT_BUDGET_CYCLES)
            return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2, int c3, int c4)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

__device__ __forceinline__ void tma_store_5d(const CUtensorMap *map, const void *src, int c0, int c1, int c2,
                                             int c3, int c4)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group"
        " [%0, {%2, %3, %4, %5, %6}], [%1];" ::"l"(reinterpret_cast<uint64_t>(map)),
        "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}

__device__ __forceinline__ void tma_store_commit_and_wait_read()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int NTHR>
__device__ __forceinline__ void block_sum2(double &a, double &b, double (*red)[32])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][w] = a;
        red[1][w] = b;
    }
    __syncthreads();
    if (w == 0) {
        constexpr int NW = NTHR / 32;
        a = lane < NW ? red[0][lane] : 0.0;
        b = lane < NW ? red[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
    }
    __syncthreads();
}

// ------------------------------------------------------- cut evaluation
// Cut values of the 2^RB basis states x0 ^ (register bits m), x0 having all
// register bits clear: v[m] = O(x0) + sum_{k in m} d_k - 2 sum_{k<k' in m} W_kk'
// where d_k is the change of O when vertex gp[k] alone flips from 0 to 1 and
// W_kk' the weight of an edge between two flipped register vertices.
template <int RB>
__device__ __forceinline__ void finish_cut(int base, const int (&d)[RB], const int (&W)[RB][RB], int (&v)[1 << RB])
{
    v[0] = base;
#pragma unroll
    for (int m = 1; m < (1 << RB); m++) {
        const int top = hibit(m);
        const int rest = m ^ (1 << top);
        int acc = v[rest] + d[top];
#pragma unroll
        for (int k2 = 0; k2 < RB; k2++)
            if (k2 < top && ((rest >> k2) & 1))
                acc -= 2 * W[top][k2];
        v[m] = acc;
    }
}

template <int RB>
__device__ __forceinline__ void eval_cost(const CostFn &f, int n, uint64_t x0, const int (&gp)[RB],
                                          int (&v)[1 << RB])
{
    int base = 0;
    for (int u = 0; u < n; u++) {
        const uint64_t nb = f.nbr[u];
        base += ((x0 >> u) & 1ull) ? __popcll(nb & ~x0) : 0;
    }
    int d[RB], W[RB][RB];
#pragma unroll
    for (int k = 0; k < RB; k++) {
        const uint64_t nb = f.nbr[gp[k]];
        d[k] = __popcll(nb) - 2 * __popcll(nb & x0);
#pragma unroll
        for (int k2 = 0; k2 < RB; k2++)
            W[k][k2] = (int)((nb >> gp[k2]) & 1ull);
    }
    finish_cut<RB>(base, d, W, v);
}

template <int RB>
__device__ __forceinline__ void eval_cut(const CutFn &f, int n, uint64_t x0, const int (&gp)[RB], int (&v)[1 << RB])
{
    int base = 0, d[RB], W[RB][RB];
#pragma unroll
    for (int k = 0; k < RB; k++) {
        d[k] = 0;
#pragma unroll
        for (int k2 = 0; k2 < RB; k2++)
            W[k][k2] = 0;
    }
    for (int c = 0; c < f.K; c++) {
        const int w = f.w[c];
        int bc = 0;
        for (int u = 0; u < n; u++) {
            const uint64_t nb = f.nbr[c][u];
            bc += ((x0 >> u) & 1ull) ? __popcll(nb & ~x0) : 0;
        }
        base += w * bc;
#pragma unroll
        for (int k = 0; k < RB; k++) {
            const uint64_t nb = f.nbr[c][gp[k]];
            d[k] += w * (__popcll(nb) - 2 * __popcll(nb & x0));
#pragma unroll
            for (int k2 = 0; k2 < RB; k2++)
                W[k][k2] += w * (int)((nb >> gp[k2]) & 1ull);
        }
    }
    finish_cut<RB>(base, d, W, v);
}

// ---------------------------------------------------------- tile geometry
// Stage plans: reg(st, k) is the local tile bit held in register slot bit k,
// thr(st, j) the local bit given by thread-index bit j (lane bits first),
// own(st) the register bits whose butterflies this stage applies. Local bits
// 0..CB-1 are the contiguous row; CB..CB+8 the high bits. swz() is the TMA
// 128-byte swizzle expressed on amplitude indices (16-byte chunk index XOR
// row mod 8). The plans are chosen so every shared-memory access of a warp is
// free of bank conflicts (16 lanes x 8 B or 8 lanes x 16 B per wavefront).
template <typename R, int NV> struct Geo;

template <int NV> struct Geo<float, NV> {
    static constexpr int CB = 4, HB = 9, T = 13, RB = 5, NTHR = 256, NST = 3;
    __host__ __device__ static constexpr int reg(int st, int k)
    {
        return st == 0 ? (k < 4 ? k : 7) : st == 1 ? 4 + k : (k == 0 ? 0 : 8 + k);
    }
    __host__ __device__ static constexpr int thr(int st, int j)
    {
        return st == 0 ? (j < 3 ? 4 + j : 5 + j) : st == 1 ? (j < 4 ? j : 5 + j) : 1 + j;
    }
    __host__ __device__ static constexpr int own(int st) { return st == 0 ? 0xF : st == 1 ? 0x1F : 0x1E; }
    __host__ __device__ static constexpr uint32_t swz(uint32_t i) { return i ^ (((i >> 4) & 7u) << 1); }
};

template <> struct Geo<double, 1> {
    static constexpr int CB = 3, HB = 9, T = 12, RB = 5, NTHR = 128, NST = 3;
    __host__ __device__ static constexpr int reg(int st, int k)
    {
        return st == 0 ? (k < 3 ? k : 3 + k) : st == 1 ? 3 + k : (k == 0 ? 0 : 7 + k);
    }
    __host__ __device__ static constexpr int thr(int st, int j)
    {
        return st == 0 ? (j < 3 ? 3 + j : 5 + j) : st == 1 ? (j < 3 ? j : 5 + j) : 1 + j;
    }
    __host__ __device__ static constexpr int own(int st) { return st == 0 ? 0x7 : st == 1 ? 0x1F : 0x1E; }
    __host__ __device__ static constexpr uint32_t swz(uint32_t i) { return i ^ ((i >> 3) & 7u); }
};

template <> struct Geo<double, 2> {
    static constexpr int CB = 3, HB = 9, T = 12, RB = 4, NTHR = 256, NST = 4;
    __host__ __device__ static constexpr int reg(int st, int k)
    {
        return st == 0 ? (k < 3 ? k : 6) : st == 1 ? 3 + k : st == 2 ? 7 + k : (k == 0 ? 11 : 2 + k);
    }
    __host__ __device__ static constexpr int thr(int st, int j)
    {
        return st == 0 ? (j < 3 ? 3 + j : 4 + j) : st == 1 ? (j < 3 ? j : 4 + j) : st == 2 ? (j < 7 ? j : 11)
                                                                                   : (j < 3 ? j : 3 + j);
    }
    __host__ __device__ static constexpr int own(int st) { return st == 0 ? 0x7 : st == 3 ? 0x1 : 0xF; }
    __host__ __device__ static constexpr uint32_t swz(uint32_t i) { return i ^ ((i >> 3) & 7u); }
};

// compile-time checks: each stage's register and thread bits partition the
// tile, and the stages' butterflies cover every tile bit exactly once.
template <typename G>
constexpr bool stages_partition()
{
    for (int st = 0; st < G::NST; st++) {
        uint32_t m = 0;
        for (int k = 0; k < G::RB; k++)
            m |= 1u << G::reg(st, k);
        for (int j = 0; j < G::T - G::RB; j++)
            m |= 1u << G::thr(st, j);
        if (m != (1u << G::T) - 1u)
            return false;
    }
    uint32_t cover = 0;
    for (int st = 0; st < G::NST; st++)
        for (int k = 0; k < G::RB; k++)
            if ((G::own(st) >> k) & 1) {
                const uint32_t bit = 1u << G::reg(st, k);
                if (cover & bit)
                    return false;
                cover |= bit;
            }
    return cover == (1u << G::T) - 1u;
}
static_assert(stages_partition<Geo<float, 1>>(), "c64 stage plan");
static_assert(stages_partition<Geo<double, 1>>(), "c128 stage plan");
static_assert(stages_partition<Geo<double, 2>>(), "c128 two-vector stage plan");

template <typename G>
__host__ __device__ constexpr uint32_t reg_offset(int st, int m)
{
    uint32_t off = 0;
    for (int k = 0; k < G::RB; k++)
        off |= (uint32_t)((m >> k) & 1) << G::reg(st, k);
    return off;
}

template <typename R, int NV, int ST>
__device__ __forceinline__ void load_regs(const typename CT<R>::T *sv, uint32_t sb,
                                          typename CT<R>::T (&a)[1 << Geo<R, NV>::RB])
{
    using G = Geo<R, NV>;
    constexpr int NR = 1 << G::RB;
    if constexpr (std::is_same<R, float>::value && G::reg(ST, 0) == 0) {
#pragma unroll
        for (int m = 0; m < NR; m += 2) {
            const float4 v = *reinterpret_cast<const float4 *>(&sv[sb ^ G::swz(reg_offset<G>(ST, m))]);
            a[m] = make_float2(v.x, v.y);
            a[m + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int m = 0; m < NR; m++)
            a[m] = sv[sb ^ G::swz(reg_offset<G>(ST, m))];
    }
}

template <typename R, int NV, int ST>
__device__ __forceinline__ void store_regs(typename CT<R>::T *sv, uint32_t sb,
                                           const typename CT<R>::T (&a)[1 << Geo<R, NV>::RB])
{
    using G = Geo<R, NV>;
    constexpr int NR = 1 << G::RB;
    if constexpr (std::is_same<R, float>::value && G::reg(ST, 0) == 0) {
#pragma unroll
        for (int m = 0; m < NR; m += 2)
            *reinterpret_cast<float4 *>(&sv[sb ^ G::swz(reg_offset<G>(ST, m))]) =
                make_float4(a[m].x, a[m].y, a[m + 1].x, a[m + 1].y);
    } else {
#pragma unroll
        for (int m = 0; m < NR; m++)
            sv[sb ^ G::swz(reg_offset<G>(ST, m))] = a[m];
    }
}

template <typename R>
struct StageCtx {
    typename CT<R>::T *sv0, *sv1;
    const typename CT<R>::T *tab;
    uint64_t fixed;
    int s, tid;
    R cb, sb;
};

// One register stage of a pass. NV = vectors carried (1: forward, 2: adjoint).
template <typename R, int NV, int ST>
__device__ __forceinline__ void run_stage(const PassArgs &A, const StageCtx<R> &X,
                                          typename CT<R>::T (&a)[1 << Geo<R, NV>::RB],
                                          typename CT<R>::T (&l)[1 << Geo<R, NV>::RB], double &acc0,
                                          double &acc1)
{
    using G = Geo<R, NV>;
    using C = typename CT<R>::T;
    constexpr int RB = G::RB, NR = 1 << RB, NTB = G::T - RB;
    constexpr bool FIRST = (ST == 0), LAST = (ST == G::NST - 1);

    uint32_t base = 0;
#pragma unroll
    for (int j = 0; j < NTB; j++)
        base |= ((uint32_t(X.tid) >> j) & 1u) << G::thr(ST, j);
    const uint32_t sb = G::swz(base);

    if (FIRST && !A.load) {
#pragma unroll
        for (int m = 0; m < NR; m++)
            a[m] = mkc<C>((R)A.amp0, (R)0);
    } else {
        load_regs<R, NV, ST>(X.sv0, sb, a);
        if constexpr (NV == 2)
            load_regs<R, NV, ST>(X.sv1, sb, l);
    }

    int gp[RB];
#pragma unroll
    for (int k = 0; k < RB; k++) {
        const int L = G::reg(ST, k);
        gp[k] = L < G::CB ? L : X.s + L - G::CB;
    }
    const uint64_t x0 = X.fixed | (uint64_t)(base & ((1u << G::CB) - 1u)) | ((uint64_t)(base >> G::CB) << X.s);

    if (FIRST && A.pre_phase) {
        int cv[NR];
        eval_cost<RB>(A.cost, A.n, x0, gp, cv);
#pragma unroll
        for (int m = 0; m < NR; m++)
            a[m] = cmul(a[m], X.tab[cv[m]]);
    }

    R gb = 0;
#pragma unroll
    for (int k = 0; k < RB; k++) {
        if (!((G::own(ST) >> k) & 1))
            continue;
        bool due = true;
        if (ST != 0)
            due = (A.hmask >> (G::reg(ST, k) - G::CB)) & 1;
        if (!due)
            continue;
#pragma unroll
        for (int m = 0; m < NR; m++) {
            if (m & (1 << k))
                continue;
            const int m1 = m | (1 << k);
            if constexpr (NV == 2) {
                gb += im_conj_mul(l[m], a[m1]) + im_conj_mul(l[m1], a[m]);
                bfly(l[m], l[m1], X.cb, X.sb);
            }
            bfly(a[m], a[m1], X.cb, X.sb);
        }
    }
    if constexpr (NV == 2)
        acc0 += (double)gb;

    bool lambda_out = false;
    if (LAST && A.post) {
        if (A.post & (POST_REDUCE | POST_LAMBDA)) {
            int ov[NR];
            eval_cut<RB>(A.obs, A.n, x0, gp, ov);
            if (A.post & POST_REDUCE) {
                R e = 0;
#pragma unroll
                for (int m = 0; m < NR; m++)
                    e += (a[m].x * a[m].x + a[m].y * a[m].y) * (R)ov[m];
                acc0 += (double)e;
            }
            if constexpr (NV == 1) {
                if (A.post & POST_LAMBDA) {
                    C lam[NR];
#pragma unroll
                    for (int m = 0; m < NR; m++)
                        lam[m] = mkc<C>(a[m].x * (R)ov[m], a[m].y * (R)ov[m]);
                    store_regs<R, NV, ST>(X.sv1, sb, lam);
                    lambda_out = true;
                }
            }
        }
        if constexpr (NV == 2) {
            if (A.post & (POST_GAMMA | POST_PHASE_CONJ)) {
                int cv[NR];
                eval_cost<RB>(A.cost, A.n, x0, gp, cv);
                if (A.post & POST_GAMMA) {
                    R g = 0;
#pragma unroll
                    for (int m = 0; m < NR; m++)
                        g += (R)cv[m] * im_conj_mul(l[m], a[m]);
                    acc1 += (double)g;
                }
                if (A.post & POST_PHASE_CONJ) {
#pragma unroll
                    for (int m = 0; m < NR; m++) {
                        const C t = X.tab[cv[m]];
                        a[m] = cmul_conj(a[m], t);
                        l[m] = cmul_conj(l[m], t);
                    }
                }
            }
        }
    }
    (void)lambda_out;
    if (!LAST || A.write) {
        store_regs<R, NV, ST>(X.sv0, sb, a);
        if constexpr (NV == 2)
            store_regs<R, NV, ST>(X.sv1, sb, l);
    }
}

// Fixed-order sum of the per-block partials by the last block to finish.
template <int NTHR>
__device__ void last_block_reduce(const PassArgs &A, double s0, double s1, double (*red)[32], unsigned tile,
                                  int b, int B)
{
    __shared__ unsigned s_last;
    const size_t plane = (size_t)B * A.tiles;
    if (threadIdx.x == 0) {
        A.partials[(size_t)b * A.tiles + tile] = s0;
        A.partials[plane + (size_t)b * A.tiles + tile] = s1;
        __threadfence();
        const unsigned total = gridDim.x * gridDim.y;
        s_last = (atomicAdd(A.counter, 1u) == total - 1u) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    for (int slot = 0; slot < 2; slot++) {
        if (A.slot_idx[slot] < 0)
            continue;
        for (int bb = 0; bb < B; bb++) {
            const double *src = A.partials + slot * plane + (size_t)bb * A.tiles;
            double a = 0.0, dummy = 0.0;
            for (int t = threadIdx.x; t < A.tiles; t += NTHR)
                a += __ldcg(src + t);
            block_sum2<NTHR>(a, dummy, red);
            if (threadIdx.x == 0)
                A.out[(size_t)bb * A.out_stride + A.slot_idx[slot]] += A.slot_scale[slot] * a;
        }
    }
    if (threadIdx.x == 0)
        *A.counter = 0u;
}

// One tiled pass over B statevectors: grid (tiles, B), one 64 KB tile per
// vector per block.
template <typename R, int NV>
__global__ void __launch_bounds__(Geo<R, NV>::NTHR)
    k_pass(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
           const __grid_constant__ PassArgs A)
{
    using G = Geo<R, NV>;
    using C = typename CT<R>::T;
    constexpr int NR = 1 << G::RB;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t bar;
    __shared__ double red[2][32];
    __shared__ int s_abort;

    const int tid = threadIdx.x;
    const int b = blockIdx.y;
    const unsigned tile = blockIdx.x;
    const int nbuf = (NV == 2 || (A.post & POST_LAMBDA)) ? 2 : 1;
    C *sv0 = reinterpret_cast<C *>(sm);
    C *sv1 = reinterpret_cast<C *>(sm + 65536);
    C *tab = reinterpret_cast<C *>(sm + nbuf * 65536);

    const int midbits = A.s - G::CB;
    const unsigned mid = tile & ((1u << midbits) - 1u);
    const unsigned hi = tile >> midbits;
    const uint64_t fixed = ((uint64_t)mid << G::CB) | ((uint64_t)hi << (A.s + G::HB));
    const int c4 = (int)(hi + (unsigned)b * ((unsigned)A.tiles >> midbits));

    if (tid == 0) {
        // a block that starts after another one timed out does no work
        s_abort = *reinterpret_cast<volatile int *>(A.err) ? 1 : 0;
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (s_abort)
        return;
    if (tid == 0 && A.load) {
        mbar_arrive_expect_tx(&bar, (uint32_t)A.nvec_io * 65536u);
        tma_load_5d(sv0, &map0, &bar, 0, (int)mid, 0, 0, c4);
        if (A.nvec_io == 2)
            tma_load_5d(sv1, &map1, &bar, 0, (int)mid, 0, 0, c4);
    }
    if (A.pre_phase || (A.post & POST_PHASE_CONJ)) {
        const C *src = reinterpret_cast<const C *>(A.tab) + ((size_t)b * A.p + A.layer) * A.tab_len;
        for (int i = tid; i < A.tab_len; i += G::NTHR)
            tab[i] = src[i];
    }
    const double2 csd = A.cs[(size_t)b * A.p + A.layer];
    StageCtx<R> X;
    X.sv0 = sv0;
    X.sv1 = sv1;
    X.tab = tab;
    X.fixed = fixed;
    X.s = A.s;
    X.tid = tid;
    X.cb = (R)csd.x;
    X.sb = (R)(A.sign_s * csd.y);

    if (A.load) {
        if (!mbar_wait_bounded(&bar, 0))
            atomicOr(&s_abort, 1);
    }
    __syncthreads();
    if (s_abort) {
        if (tid == 0) {
            atomicExch(A.err, 1);
            mbar_wait_bounded(&bar, 0);
        }
        return;
    }

    C a[NR], l[NR];
    double acc0 = 0.0, acc1 = 0.0;
    if (A.is_low) {
        run_stage<R, NV, 0>(A, X, a, l, acc0, acc1);
        __syncthreads();
    }
    run_stage<R, NV, 1>(A, X, a, l, acc0, acc1);
    __syncthreads();
    run_stage<R, NV, 2>(A, X, a, l, acc0, acc1);
    if constexpr (G::NST == 4) {
        __syncthreads();
        run_stage<R, NV, 3>(A, X, a, l, acc0, acc1);
    }

    if (A.write) {
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_5d(&map0, sv0, 0, (int)mid, 0, 0, c4);
            if (nbuf == 2)
                tma_store_5d(&map1, sv1, 0, (int)mid, 0, 0, c4);
            tma_store_commit_and_wait_read();
        }
    }
    if (A.slot_idx[0] >= 0 || A.slot_idx[1] >= 0) {
        block_sum2<G::NTHR>(acc0, acc1, red);
        last_block_reduce<G::NTHR>(A, acc0, acc1, red, tile, b, gridDim.y);
    }
}

// ------------------------------------------------------ parameter tables
// T_l[c] = exp(-i ((gamma_l c) mod 2 pi)) for c = 0..tab_len-1, in FP64 then
// rounded once to the amplitude precision; (cos beta_l, sin beta_l) in FP64.
template <typename R>
__global__ void k_params(int B, int p, int tab_len, const double *__restrict__ gamma,
                         const double *__restrict__ beta, typename CT<R>::T *__restrict__ tab,
                         double2 *__restrict__ cs)
{
    const double TWO_PI = 6.283185307179586476925286766559;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)B * p * tab_len;
    if (i < total) {
        const long long bl = i / tab_len;
        const int c = (int)(i - bl * tab_len);
        double ang = fmod(gamma[bl] * (double)c, TWO_PI);
        if (ang < 0.0)
            ang += TWO_PI;
        double sn, cn;
        sincos(ang, &sn, &cn);
        tab[i] = mkc<typename CT<R>::T>((R)cn, (R)(-sn));
    }
    if (i < (long long)B * p) {
        double sn, cn;
        sincos(beta[i], &sn, &cn);
        cs[i] = make_double2(cn, sn);
    }
}

// --------------------------------------------- whole circuit in one CTA
__device__ __forceinline__ int cost_direct(const CostFn &f, int n, uint32_t x)
{
    int c = 0;
    for (int u = 0; u < n; u++)
        c += ((x >> u) & 1u) ? __popcll(f.nbr[u] & ~(uint64_t)x) : 0;
    return c;
}

__device__ __forceinline__ int cut_direct(const CutFn &f, int n, uint32_t x)
{
    int v = 0;
    for (int c = 0; c < f.K; c++) {
        int s = 0;
        for (int u = 0; u < n; u++)
            s += ((x >> u) & 1u) ? __popcll(f.nbr[c][u] & ~(uint64_t)x) : 0;
        v += f.w[c] * s;
    }
    return v;
}

template <typename R>
__global__ void __launch_bounds__(256) k_small(const __grid_constant__ SmallArgs A)
{
    using C = typename CT<R>::T;
    constexpr int NT = 256;
    extern __shared__ unsigned char smem_raw[];
    __shared__ double red[2][32];
    const int n = A.n, N = 1 << n, half = N >> 1, b = blockIdx.x, tid = threadIdx.x;
    C *phi = reinterpret_cast<C *>(smem_raw);
    C *lam = phi + N;
    C *tab = phi + (A.mode == SMALL_GRAD ? 2 * N : N);

    for (int x = tid; x < N; x += NT)
        phi[x] = mkc<C>((R)A.amp0, (R)0);
    for (int l = 0; l < A.p; l++) {
        __syncthreads();
        const C *src = reinterpret_cast<const C *>(A.tab) + ((size_t)b * A.p + l) * A.tab_len;
        for (int i = tid; i < A.tab_len; i += NT)
            tab[i] = src[i];
        const double2 cs = A.cs[(size_t)b * A.p + l];
        const R c = (R)cs.x, s = (R)cs.y;
        __syncthreads();
        for (int x = tid; x < N; x += NT)
            phi[x] = cmul(phi[x], tab[cost_direct(A.cost, n, (uint32_t)x)]);
        for (int q = 0; q < n; q++) {
            __syncthreads();
            for (int j = tid; j < half; j += NT) {
                const int x0 = ((j >> q) << (q + 1)) | (j & ((1 << q) - 1));
                bfly(phi[x0], phi[x0 | (1 << q)], c, s);
            }
        }
    }
    __syncthreads();
    if (A.write_state) {
        C *dst = reinterpret_cast<C *>(A.state) + (size_t)b * N;
        for (int x = tid; x < N; x += NT)
            dst[x] = phi[x];
    }
    double e = 0.0, dummy = 0.0;
    for (int x = tid; x < N; x += NT)
        e += (double)((phi[x].x * phi[x].x + phi[x].y * phi[x].y) * (R)cut_direct(A.obs, n, (uint32_t)x));
    block_sum2<NT>(e, dummy, red);
    if (tid == 0)
        A.out[(size_t)b * A.out_stride] = e;
    if (A.mode != SMALL_GRAD)
        return;

    for (int x = tid; x < N; x += NT) {
        const R o = (R)cut_direct(A.obs, n, (uint32_t)x);
        lam[x] = mkc<C>(phi[x].x * o, phi[x].y * o);
    }
    for (int l = A.p - 1; l >= 0; l--) {
        const double2 cs = A.cs[(size_t)b * A.p + l];
        const R c = (R)cs.x, s = (R)(-cs.y);
        double gb = 0.0, gg = 0.0;
        for (int q = 0; q < n; q++) {
            __syncthreads();
            for (int j = tid; j < half; j += NT) {
                const int x0 = ((j >> q) << (q + 1)) | (j & ((1 << q) - 1));
                const int x1 = x0 | (1 << q);
                gb += (double)(im_conj_mul(lam[x0], phi[x1]) + im_conj_mul(lam[x1], phi[x0]));
                bfly(phi[x0], phi[x1], c, s);
                bfly(lam[x0], lam[x1], c, s);
            }
        }
        __syncthreads();
        if (l > 0) {
            const C *src = reinterpret_cast<const C *>(A.tab) + ((size_t)b * A.p + l) * A.tab_len;
            for (int i = tid; i < A.tab_len; i += NT)
                tab[i] = src[i];
        }
        __syncthreads();
        for (int x = tid; x < N; x += NT) {
            const int cv = cost_direct(A.cost, n, (uint32_t)x);
            gg += (double)((R)cv * im_conj_mul(lam[x], phi[x]));
            if (l > 0) {
                const C t = tab[cv];
                phi[x] = cmul_conj(phi[x], t);
                lam[x] = cmul_conj(lam[x], t);
            }
        }
        block_sum2<NT>(gb, gg, red);
        if (tid == 0) {
            A.out[(size_t)b * A.out_stride + 1 + l] = 2.0 * gg;
            A.out[(size_t)b * A.out_stride + 1 + A.p + l] = 2.0 * gb;
        }
    }
}

// -------------------------------------------- aggregation over a state
// A warp handles 1024-amplitude chunks. For C64 a lane holds 32 amplitudes
// whose index bits 0 and 6..9 vary (float4 loads: 512 contiguous bytes per
// warp instruction); for C128 bits 5..9 vary (double2 loads).
template <typename R> struct AggLayout;
template <> struct AggLayout<float> {
    __host__ __device__ static constexpr int gp(int k) { return k == 0 ? 0 : 5 + k; }
    __device__ static uint64_t lane_bits(int lane) { return (uint64_t)lane << 1; }
    __device__ static void load(const float2 *s, uint64_t base, int lane, float2 (&a)[32])
    {
        const float4 *p = reinterpret_cast<const float4 *>(s + base) + lane;
#pragma unroll
        for (int i = 0; i < 16; i++) {
            const float4 v = __ldcs(p + 32 * i);
            a[2 * i] = make_float2(v.x, v.y);
            a[2 * i + 1] = make_float2(v.z, v.w);
        }
    }
};
template <> struct AggLayout<double> {
    __host__ __device__ static constexpr int gp(int k) { return 5 + k; }
    __device__ static uint64_t lane_bits(int lane) { return (uint64_t)lane; }
    __device__ static void load(const double2 *s, uint64_t base, int lane, double2 (&a)[32])
    {
        const double2 *p = s + base + lane;
#pragma unroll
        for (int i = 0; i < 32; i++)
            a[i] = __ldcs(p + 32 * i);
    }
};

template <int NTHR>
__device__ void agg_finish(const AggArgs &A, int nslots, double (*vals), double (*red)[32])
{
    // vals[t]: this block's partial of slot t (already block-reduced, valid in thread 0)
    __shared__ unsigned s_last;
    if (threadIdx.x == 0) {
        for (int t = 0; t < nslots; t++)
            A.partials[(size_t)t * gridDim.x + blockIdx.x] = vals[t];
        __threadfence();
        s_last = (atomicAdd(A.counter, 1u) == gridDim.x - 1u) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    for (int t = 0; t < nslots; t++) {
        double a = 0.0, dummy = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += NTHR)
            a += __ldcg(A.partials + (size_t)t * gridDim.x + i);
        block_sum2<NTHR>(a, dummy, red);
        if (threadIdx.x == 0) {
            if (A.num_terms == 0) {
                *A.out_energy += a;
            } else {
                if (A.out_terms)
                    A.out_terms[t] = a;
                *A.out_energy += A.term_w[t] * 0.5 * (1.0 - a);
            }
        }
    }
    if (threadIdx.x == 0)
        *A.counter = 0u;
}

// E += sum_x |psi_x|^2 O(x) over a stored state (one read).
template <typename R>
__global__ void __launch_bounds__(256) k_agg_fused(const __grid_constant__ AggArgs A)
{
    using C = typename CT<R>::T;
    using L = AggLayout<R>;
    __shared__ double red[2][32];
    const int lane = threadIdx.x & 31;
    const C *st = reinterpret_cast<const C *>(A.state);
    double acc = 0.0;
    if (A.n < 10) {
        const int N = 1 << A.n;
        if (blockIdx.x == 0)
            for (int x = threadIdx.x; x < N; x += 256)
                acc += (double)((st[x].x * st[x].x + st[x].y * st[x].y) * (R)cut_direct(A.obs, A.n, (uint32_t)x));
    } else {
        int gp[5];
#pragma unroll
        for (int k = 0; k < 5; k++)
            gp[k] = L::gp(k);
        const uint64_t warps = (uint64_t)gridDim.x * 8;
        for (uint64_t ch = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5); ch < A.chunks; ch += warps) {
            C a[32];
            L::load(st, ch << 10, lane, a);
            int ov[32];
            eval_cut<5>(A.obs, A.n, (ch << 10) | L::lane_bits(lane), gp, ov);
            R e = 0;
#pragma unroll
            for (int m = 0; m < 32; m++)
                e += (a[m].x * a[m].x + a[m].y * a[m].y) * (R)ov[m];
            acc += (double)e;
        }
    }
    double dummy = 0.0;
    block_sum2<256>(acc, dummy, red);
    double v[1] = {acc};
    agg_finish<256>(A, 1, v, red);
}

// Per-term <Z_u Z_v> over a stored state, all terms of the launch in one read.
// Per lane: p_m = |psi_m|^2 for its 32 amplitudes, Walsh-Hadamard transformed
// over the 5 register bits, F[mask] = sum_m p_m (-1)^{popcount(m & mask)};
// a term whose endpoints fall on register bits `mask` (and on lane/chunk bits
// elsewhere) contributes sign(x0) * F[mask].
template <typename R>
__global__ void __launch_bounds__(256) k_agg_terms(const __grid_constant__ AggArgs A)
{
    using C = typename CT<R>::T;
    using L = AggLayout<R>;
    extern __shared__ double acc_s[];  // [num_terms][256]
    __shared__ double red[2][32];
    const int lane = threadIdx.x & 31, T = A.num_terms;
    for (int t = 0; t < T; t++)
        acc_s[t * 256 + threadIdx.x] = 0.0;
    const C *st = reinterpret_cast<const C *>(A.state);
    if (A.n < 10) {
        const int N = 1 << A.n;
        if (blockIdx.x == 0)
            for (int x = threadIdx.x; x < N; x += 256) {
                const double pr = (double)(st[x].x * st[x].x + st[x].y * st[x].y);
                for (int t = 0; t < T; t++)
                    acc_s[t * 256 + threadIdx.x] += (((x >> A.term_u[t]) ^ (x >> A.term_v[t])) & 1) ? -pr : pr;
            }
    } else {
        // register-bit masks of each term's endpoints
        uint32_t tmask[64];
        uint64_t tfix[64];
        for (int t = 0; t < T; t++) {
            uint32_t m = 0;
            uint64_t f = 0;
            const int ends[2] = {A.term_u[t], A.term_v[t]};
            for (int e = 0; e < 2; e++) {
                int k = -1;
#pragma unroll
                for (int kk = 0; kk < 5; kk++)
                    if (L::gp(kk) == ends[e])
                        k = kk;
                if (k >= 0)
                    m ^= 1u << k;
                else
                    f ^= 1ull << ends[e];
            }
            tmask[t] = m;
            tfix[t] = f;
        }
        const uint64_t warps = (uint64_t)gridDim.x * 8;
        for (uint64_t ch = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5); ch < A.chunks; ch += warps) {
            C a[32];
            L::load(st, ch << 10, lane, a);
            R F[32];
#pragma unroll
            for (int m = 0; m < 32; m++)
                F[m] = a[m].x * a[m].x + a[m].y * a[m].y;
#pragma unroll
            for (int k = 0; k < 5; k++)
#pragma unroll
                for (int m = 0; m < 32; m++)
                    if (!(m & (1 << k))) {
                        const R u = F[m], v = F[m | (1 << k)];
                        F[m] = u + v;
                        F[m | (1 << k)] = u - v;
                    }
            const uint64_t x0 = (ch << 10) | L::lane_bits(lane);
            for (int t = 0; t < T; t++) {
                R f = F[0];
#pragma unroll
                for (int q = 1; q < 32; q++)
                    f = (tmask[t] == (uint32_t)q) ? F[q] : f;
                const R sgn = (__popcll(x0 & tfix[t]) & 1) ? (R)-1 : (R)1;
                acc_s[t * 256 + threadIdx.x] += (double)(sgn * f);
            }
        }
    }
    double vals[64];
    for (int t = 0; t < T; t++) {
        double v = acc_s[t * 256 + threadIdx.x], dummy = 0.0;
        block_sum2<256>(v, dummy, red);
        vals[t] = v;
    }
    agg_finish<256>(A, T, vals, red);
}

// ------------------------------------------------------------- launchers
int tile_bits(bool c128) { return c128 ? Geo<double, 1>::T : Geo<float, 1>::T; }

size_t pass_smem_bytes(bool c128, int nbuf)
{
    return (size_t)nbuf * 65536 + (size_t)MAXTAB * (c128 ? 16 : 8) + 1024;
}

int launch_params(bool c128, int B, int p, int tab_len, const double *d_gamma, const double *d_beta, void *d_tab,
                  double2 *d_cs, cudaStream_t st)
{
    const long long total = (long long)B * p * (tab_len > 1 ? tab_len : 1);
    const int grid = (int)((total + 255) / 256);
    if (c128)
        k_params<double><<<grid, 256, 0, st>>>(B, p, tab_len, d_gamma, d_beta, (double2 *)d_tab, d_cs);
    else
        k_params<float><<<grid, 256, 0, st>>>(B, p, tab_len, d_gamma, d_beta, (float2 *)d_tab, d_cs);
    return (int)cudaGetLastError();
}

template <typename R, int NV>
static int launch_pass_t(int nbuf, const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int B,
                         cudaStream_t st)
{
    const size_t smem = pass_smem_bytes(sizeof(R) == 8, nbuf);
    static bool attr_done[3] = {false, false, false};
    if (!attr_done[nbuf]) {
        cudaError_t e = cudaFuncSetAttribute(k_pass<R, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return (int)e;
        attr_done[nbuf] = true;
    }
    dim3 grid((unsigned)a.tiles, (unsigned)B);
    k_pass<R, NV><<<grid, Geo<R, NV>::NTHR, smem, st>>>(m0, m1, a);
    return (int)cudaGetLastError();
}

int launch_pass(bool c128, int nv_kernel, int nbuf, const CUtensorMap &m0, const CUtensorMap &m1,
                const PassArgs &a, int B, cudaStream_t st)
{
    if (c128)
        return nv_kernel == 2 ? launch_pass_t<double, 2>(nbuf, m0, m1, a, B, st)
                              : launch_pass_t<double, 1>(nbuf, m0, m1, a, B, st);
    return nv_kernel == 2 ? launch_pass_t<float, 2>(nbuf, m0, m1, a, B, st)
                          : launch_pass_t<float, 1>(nbuf, m0, m1, a, B, st);
}

size_t small_smem_bytes(bool c128, int n, int mode)
{
    const size_t amp = c128 ? 16 : 8;
    return ((mode == SMALL_GRAD ? 2 : 1) * ((size_t)1 << n) + MAXTAB) * amp;
}

int small_max_qubits(bool c128, int mode)
{
    // largest n whose state(s) plus the phase table fit the opt-in shared memory
    int n = 1;
    while (n < 20 && small_smem_bytes(c128, n + 1, mode) <= 200 * 1024)
        n++;
    return n;
}

int launch_small(bool c128, const SmallArgs &a, int B, cudaStream_t st)
{
    const size_t smem = small_smem_bytes(c128, a.n, a.mode);
    cudaError_t e;
    if (c128) {
        e = cudaFuncSetAttribute(k_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return (int)e;
        k_small<double><<<B, 256, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return (int)e;
        k_small<float><<<B, 256, smem, st>>>(a);
    }
    return (int)cudaGetLastError();
}

int agg_grid(bool c128)
{
    (void)c128;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * 4;
}

int launch_agg_fused(bool c128, const AggArgs &a, cudaStream_t st, int grid)
{
    if (c128)
        k_agg_fused<double><<<grid, 256, 0, st>>>(a);
    else
        k_agg_fused<float><<<grid, 256, 0, st>>>(a);
    return (int)cudaGetLastError();
}

int launch_agg_terms(bool c128, const AggArgs &a, cudaStream_t st, int grid)
{
    const size_t smem = (size_t)a.num_terms * 256 * sizeof(double);
    cudaError_t e;
    if (c128) {
        e = cudaFuncSetAttribute(k_agg_terms<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 256 * 8);
        if (e != cudaSuccess)
            return (int)e;
        k_agg_terms<double><<<grid, 256, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_agg_terms<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 256 * 8);
        if (e != cudaSuccess)
            return (int)e;
        k_agg_terms<float><<<grid, 256, smem, st>>>(a);
    }
    return (int)cudaGetLastError();
}

}  // namespace aaq

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

// The tiled passes keep the statevector in the twisted frame
//   psi~(x) = i^|x| psi(x)        (|x| = number of one bits of x).
// There RX(2 beta) on the pair (x, x ^ e_q), x_q = 0, is the real rotation
//   (a, b) <- (c a - s b, c b + s a)
// applied to real and imaginary parts alike, so one packed two-lane FMA
// updates a whole complex amplitude. Up to the real factor f it reads
//   f = cos beta, t = tan beta:            (a, b) <- (a - t b, b + t a)
// and for |sin| > |cos| the same form with f = sin beta, t = -cot beta is the
// rotation by beta - pi/2, i.e. RX(2 beta) with the factor -i X dropped on
// every qubit. (-i X)^n commutes with the phase and the observable (a cut
// value is invariant when all bits flip), so energies and gradients are
// unchanged; only the exported statevector is corrected for it.
template <typename C, typename R>
__device__ __forceinline__ void rot(C &a, C &b, R t)
{
    if constexpr (std::is_same<R, float>::value) {
        const float2 a0 = a;
        a = __ffma2_rn(make_float2(-t, -t), b, a);
        b = __ffma2_rn(make_float2(t, t), a0, b);
    } else {
        const C a0 = a;
        a.x = fma(-t, b.x, a.x);
        a.y = fma(-t, b.y, a.y);
        b.x = fma(t, a0.x, b.x);
        b.y = fma(t, a0.y, b.y);
    }
}

// (a, b) <- (t a - b, t b + a): the same twisted-frame rotation by beta with
// the factor f = sin beta dropped instead (t = cot beta). Ising plans use it
// when |sin| > |cos|: with fields the cost no longer commutes with X^n, so
// the -iX factor that the shifted form drops cannot be dropped there.
template <typename C, typename R>
__device__ __forceinline__ void rotc(C &a, C &b, R t)
{
    if constexpr (std::is_same<R, float>::value) {
        const float2 a0 = a;
        a = __ffma2_rn(make_float2(t, t), a0, make_float2(-b.x, -b.y));
        b = __ffma2_rn(make_float2(t, t), b, a0);
    } else {
        const C a0 = a;
        a.x = fma(t, a0.x, -b.x);
        a.y = fma(t, a0.y, -b.y);
        b.x = fma(t, b.x, a0.x);
        b.y = fma(t, b.y, a0.y);
    }
}

// exp(i theta) for a phase angle given in FP64: reduced mod 2 pi in FP64,
// then cos/sin in the amplitude precision (the reduced argument is exact to
// the rounding of a float in [0, 2 pi)).
template <typename R>
__device__ __forceinline__ typename CT<R>::T unit_phase(double theta)
{
    const double TWO_PI = 6.283185307179586476925286766559;
    const double a = theta - TWO_PI * floor(theta * (1.0 / TWO_PI));  // in [0, 2 pi)
    typename CT<R>::T z;
    if constexpr (std::is_same<R, float>::value) {
        float sn, cn;
        sincosf((float)a, &sn, &cn);
        z.x = cn;
        z.y = sn;
    } else {
        double sn, cn;
        sincos(a, &sn, &cn);
        z.x = cn;
        z.y = sn;
    }
    return z;
}

// acc += (u.x v.x, u.y v.y): Re(conj(u) v) summed over the two lanes later
template <typename C>
__device__ __forceinline__ void dot_acc(C &acc, const C &u, const C &v)
{
    if constexpr (std::is_same<C, float2>::value) {
        acc = __ffma2_rn(u, v, acc);
    } else {
        acc.x = fma(u.x, v.x, acc.x);
        acc.y = fma(u.y, v.y, acc.y);
    }
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
// A tile holds 2^T amplitudes per vector: local bits 0..CB-1 are one 128-byte
// row of contiguous amplitudes, local bits CB..CB+HB-1 are HB consecutive
// qubits s..s+HB-1 (rows at stride 2^s). NSTAGE tiles are in flight per CTA.
// Register stages: reg(st, k) is the local bit held in register-slot bit k,
// thr(st, j) the local bit given by thread-index bit j (lane bits first),
// own(st) the register bits whose butterflies stage st applies. swz() is the
// TMA 128-byte swizzle on amplitude indices (16-byte chunk XOR row mod 8).
// Every plan keeps each warp's shared-memory accesses free of bank conflicts
// (16 lanes x 8 B or 8 lanes x 16 B per wavefront).
template <typename R, int NV> struct Geo;

// complex64, one vector: 64 KB tiles (13 qubits), 32 amplitudes per thread
template <> struct Geo<float, 1> {
    static constexpr int CB = 4, HB = 9, T = 13, RB = 5, NTHR = 256, NST = 3, NSTAGE = 3;
    static constexpr int MAXREG = 168;  // 9 warps: 3 share a sub-partition's 16K registers
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

// complex64, two vectors (adjoint): 2 x 32 KB tiles (12 qubits), 16 per thread.
// Stage 3 exists only in the cluster pass: the stage-2 layout again, whose
// register bits 2, 3 (local bits 10, 11) then hold the cluster's qubits.
template <> struct Geo<float, 2> {
    static constexpr int CB = 4, HB = 8, T = 12, RB = 4, NTHR = 256, NST = 3, NSTAGE = 3;
    static constexpr int MAXREG = 168;  // 9 warps: 3 share a sub-partition's 16K registers
    __host__ __device__ static constexpr int reg(int st, int k) { return st == 0 ? k : st == 1 ? 4 + k : 8 + k; }
    __host__ __device__ static constexpr int thr(int st, int j)
    {
        return st == 0 ? 4 + j : st == 1 ? (j < 4 ? j : 4 + j) : j;
    }
    __host__ __device__ static constexpr int own(int st) { return st == 3 ? 0xC : 0xF; }
    __host__ __device__ static constexpr uint32_t swz(uint32_t i) { return i ^ (((i >> 4) & 7u) << 1); }
};

// complex128, one vector: 64 KB tiles (12 qubits), 32 amplitudes per thread
template <> struct Geo<double, 1> {
    static constexpr int CB = 3, HB = 9, T = 12, RB = 5, NTHR = 128, NST = 3, NSTAGE = 3;
    static constexpr int MAXREG = 255;  // 5 warps: at most 2 per sub-partition
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

// complex128, two vectors (adjoint): 2 x 32 KB tiles (11 qubits), 16 per thread
template <> struct Geo<double, 2> {
    static constexpr int CB = 3, HB = 8, T = 11, RB = 4, NTHR = 128, NST = 3, NSTAGE = 3;
    static constexpr int MAXREG = 255;  // 5 warps: at most 2 per sub-partition
    __host__ __device__ static constexpr int reg(int st, int k)
    {
        return st == 0 ? (k < 3 ? k : 6) : st == 1 ? 3 + k : 7 + k;
    }
    __host__ __device__ static constexpr int thr(int st, int j)
    {
        return st == 0 ? (j < 3 ? 3 + j : 4 + j) : st == 1 ? (j < 3 ? j : 4 + j) : j;
    }
    __host__ __device__ static constexpr int own(int st) { return st == 0 ? 0x7 : 0xF; }
    __host__ __device__ static constexpr uint32_t swz(uint32_t i) { return i ^ ((i >> 3) & 7u); }
};

// compile-time checks: each stage's register and thread bits partition the
// tile, the stages' butterflies cover every tile bit exactly once, and the
// pipeline fits the 227 KB of shared memory.
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
    return cover == (1u << G::T) - 1u && G::CB + G::HB == G::T && (1 << (G::T - G::RB)) == G::NTHR;
}
static_assert(stages_partition<Geo<float, 1>>(), "c64 stage plan");
static_assert(stages_partition<Geo<float, 2>>(), "c64 two-vector stage plan");
static_assert(stages_partition<Geo<double, 1>>(), "c128 stage plan");
static_assert(stages_partition<Geo<double, 2>>(), "c128 two-vector stage plan");

template <typename R, int NV>
__host__ __device__ constexpr size_t tile_bytes() { return ((size_t)1 << Geo<R, NV>::T) * sizeof(R) * 2; }

// shared memory of one pass CTA: pipeline buffers, phase table, cut masks;
// for Ising plans (IS) pipeline buffers, per-thread values of both functions
// and per-thread cost phases
template <typename R, int NV, bool IS = false>
__host__ __device__ constexpr size_t pass_smem_total()
{
    using G = Geo<R, NV>;
    return IS ? (size_t)G::NSTAGE * NV * tile_bytes<R, NV>() + (size_t)4 * (G::RB + 1) * G::NTHR * sizeof(R) + 1024
              : (size_t)G::NSTAGE * NV * tile_bytes<R, NV>() + 2 * (size_t)MAXTAB * sizeof(R) * 2 +
                    (size_t)(2 * MAXK) * MAXN * 8 + 1024;
}
// static shared memory of the pass kernel (mbarriers, per-point sums, cut
// constants) plus slack for the final reduction's flag
template <typename R, int NV, bool IS = false>
__host__ __device__ constexpr size_t pass_static_smem()
{
    using G = Geo<R, NV>;
    return IS ? 2 * G::NSTAGE * 8 + 2 * 3 * 32 * 8 + 4 + 2 * MAXK * 4 + 4 + 4 + 2 * 2 * 2 * 32 * 4 +
                    G::NSTAGE * 2 * 16 * sizeof(R) + G::NSTAGE * 16 * 2 * sizeof(R) + 2 * 32 * sizeof(R) +
                    2 * 32 * 2 * sizeof(R) + 2 * MAXN * 8 + 256
              : 2 * G::NSTAGE * 8 + 2 * 3 * 32 * 8 + 4 + 2 * MAXK * 4 + G::NSTAGE * 2 * 16 * 4 +
                    2 * (G::RB + 1) * G::NTHR * 4 + 2 * 2 * 2 * 32 * 4 + 256;
}
static_assert(pass_smem_total<float, 1>() + pass_static_smem<float, 1>() <= 227 * 1024, "c64 pipeline smem");
static_assert(pass_smem_total<float, 2>() + pass_static_smem<float, 2>() <= 227 * 1024, "c64 adjoint pipeline smem");
static_assert(pass_smem_total<double, 1>() + pass_static_smem<double, 1>() <= 227 * 1024, "c128 pipeline smem");
static_assert(pass_smem_total<double, 2>() + pass_static_smem<double, 2>() <= 227 * 1024,
              "c128 adjoint pipeline smem");
static_assert(pass_smem_total<float, 1, true>() + pass_static_smem<float, 1, true>() <= 227 * 1024, "Ising smem");
static_assert(pass_smem_total<float, 2, true>() + pass_static_smem<float, 2, true>() <= 227 * 1024, "Ising smem");
static_assert(pass_smem_total<double, 1, true>() + pass_static_smem<double, 1, true>() <= 227 * 1024, "Ising smem");
static_assert(pass_smem_total<double, 2, true>() + pass_static_smem<double, 2, true>() <= 227 * 1024, "Ising smem");

template <typename G>
__host__ __device__ constexpr uint32_t reg_offset(int st, int m)
{
    uint32_t off = 0;
    for (int k = 0; k < G::RB; k++)
        off |= (uint32_t)((m >> k) & 1) << G::reg(st, k);
    return off;
}

// Shared-memory index of register m in stage ST: sb ^ K_m, sb = swz(thread
// bits), K_m = swz(register bits of m). Only the bits in LOW (those sb and
// some K_m can both have: the swizzle's target bits) need the XOR; the rest
// add. So sb ^ K_m = (sb & ~LOW) + (K_m & ~LOW) + ((sb & LOW) ^ (K_m & LOW)):
// at most 2^|LOW| distinct bases per stage, each access a compile-time
// offset from one of them (checked below for every thread and register).
template <typename G, int ST>
__host__ __device__ constexpr uint32_t split_low()
{
    uint32_t sbits = 0, kbits = 0;
    for (int j = 0; j < G::T - G::RB; j++)
        sbits |= G::swz(1u << G::thr(ST, j));
    for (int k = 0; k < G::RB; k++)
        kbits |= G::swz(1u << G::reg(ST, k));
    return sbits & kbits;
}
template <typename G, int ST>
__device__ __forceinline__ uint32_t smem_index(uint32_t sbh, uint32_t sbl, int m)
{
    constexpr uint32_t LOW = split_low<G, ST>();
    const uint32_t K = G::swz(reg_offset<G>(ST, m));
    return (sbh + (sbl ^ (K & LOW))) + (K & ~LOW);
}
template <typename G, int ST>
constexpr bool split_ok()
{
    constexpr int NTB = G::T - G::RB;
    constexpr uint32_t LOW = split_low<G, ST>();
    for (uint32_t tid = 0; tid < (1u << NTB); tid++) {
        uint32_t base = 0;
        for (int j = 0; j < NTB; j++)
            base |= ((tid >> j) & 1u) << G::thr(ST, j);
        const uint32_t sb = G::swz(base);
        for (int m = 0; m < (1 << G::RB); m++) {
            const uint32_t K = G::swz(reg_offset<G>(ST, m));
            if ((sb ^ K) != (sb & ~LOW) + (K & ~LOW) + ((sb & LOW) ^ (K & LOW)))
                return false;
        }
    }
    return true;
}
static_assert(split_ok<Geo<float, 1>, 0>() && split_ok<Geo<float, 1>, 1>() && split_ok<Geo<float, 1>, 2>() &&
                  split_ok<Geo<float, 2>, 0>() && split_ok<Geo<float, 2>, 1>() && split_ok<Geo<float, 2>, 2>() &&
                  split_ok<Geo<double, 1>, 0>() && split_ok<Geo<double, 1>, 1>() && split_ok<Geo<double, 1>, 2>() &&
                  split_ok<Geo<double, 2>, 0>() && split_ok<Geo<double, 2>, 1>() && split_ok<Geo<double, 2>, 2>(),
              "shared-memory index split");

template <typename R, int NV, int ST>
__device__ __forceinline__ void load_regs(const typename CT<R>::T *sv, uint32_t sb,
                                          typename CT<R>::T (&a)[1 << Geo<R, NV>::RB])
{
    using G = Geo<R, NV>;
    constexpr int NR = 1 << G::RB;
    constexpr uint32_t LOW = split_low<G, ST>();
    const uint32_t sbh = sb & ~LOW, sbl = sb & LOW;
    if constexpr (std::is_same<R, float>::value && G::reg(ST, 0) == 0) {
#pragma unroll
        for (int m = 0; m < NR; m += 2) {
            const float4 v = *reinterpret_cast<const float4 *>(&sv[smem_index<G, ST>(sbh, sbl, m)]);
            a[m] = make_float2(v.x, v.y);
            a[m + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int m = 0; m < NR; m++)
            a[m] = sv[smem_index<G, ST>(sbh, sbl, m)];
    }
}

template <typename R, int NV, int ST>
__device__ __forceinline__ void store_regs(typename CT<R>::T *sv, uint32_t sb,
                                           const typename CT<R>::T (&a)[1 << Geo<R, NV>::RB])
{
    using G = Geo<R, NV>;
    constexpr int NR = 1 << G::RB;
    constexpr uint32_t LOW = split_low<G, ST>();
    const uint32_t sbh = sb & ~LOW, sbl = sb & LOW;
    if constexpr (std::is_same<R, float>::value && G::reg(ST, 0) == 0) {
#pragma unroll
        for (int m = 0; m < NR; m += 2)
            *reinterpret_cast<float4 *>(&sv[smem_index<G, ST>(sbh, sbl, m)]) =
                make_float4(a[m].x, a[m].y, a[m + 1].x, a[m + 1].y);
    } else {
#pragma unroll
        for (int m = 0; m < NR; m++)
            sv[smem_index<G, ST>(sbh, sbl, m)] = a[m];
    }
}

// The local index bits a thread's index gives in stage ST, as runs of
// consecutive thread bits that move by one shift: base = OR of
// (tid & mask) << shift (a right shift for negative shifts).
struct BitRuns {
    int n;
    uint32_t mask[16];
    int shift[16];
};
template <typename G, int ST>
__host__ __device__ constexpr BitRuns stage_runs()
{
    BitRuns r{0, {}, {}};
    constexpr int NTB = G::T - G::RB;
    int j = 0;
    while (j < NTB) {
        const int d = G::thr(ST, j) - j;
        int e = j + 1;
        while (e < NTB && G::thr(ST, e) - e == d)
            e++;
        r.mask[r.n] = ((1u << e) - 1u) & ~((1u << j) - 1u);
        r.shift[r.n] = d;
        r.n++;
        j = e;
    }
    return r;
}
template <typename G, int ST>
__device__ __forceinline__ uint32_t stage_base(uint32_t tid)
{
    constexpr BitRuns R = stage_runs<G, ST>();
    uint32_t base = 0;
#pragma unroll
    for (int i = 0; i < R.n; i++)
        base |= R.shift[i] >= 0 ? (tid & R.mask[i]) << R.shift[i] : (tid & R.mask[i]) >> -R.shift[i];
    return base;
}
template <typename G, int ST>
constexpr bool stage_runs_ok()
{  // the runs reproduce the bit-by-bit map for every thread index
    constexpr int NTB = G::T - G::RB;
    constexpr BitRuns R = stage_runs<G, ST>();
    for (uint32_t tid = 0; tid < (1u << NTB); tid++) {
        uint32_t a = 0, b = 0;
        for (int j = 0; j < NTB; j++)
            a |= ((tid >> j) & 1u) << G::thr(ST, j);
        for (int i = 0; i < R.n; i++)
            b |= R.shift[i] >= 0 ? (tid & R.mask[i]) << R.shift[i] : (tid & R.mask[i]) >> -R.shift[i];
        if (a != b)
            return false;
    }
    return true;
}
static_assert(stage_runs_ok<Geo<float, 1>, 0>() && stage_runs_ok<Geo<float, 1>, 1>() &&
                  stage_runs_ok<Geo<float, 1>, 2>(), "c64 thread-bit runs");
static_assert(stage_runs_ok<Geo<float, 2>, 0>() && stage_runs_ok<Geo<float, 2>, 1>() &&
                  stage_runs_ok<Geo<float, 2>, 2>(), "c64 two-vector thread-bit runs");
static_assert(stage_runs_ok<Geo<double, 1>, 0>() && stage_runs_ok<Geo<double, 1>, 1>() &&
                  stage_runs_ok<Geo<double, 1>, 2>(), "c128 thread-bit runs");
static_assert(stage_runs_ok<Geo<double, 2>, 0>() && stage_runs_ok<Geo<double, 2>, 1>() &&
                  stage_runs_ok<Geo<double, 2>, 2>(), "c128 two-vector thread-bit runs");

// A cut function as neighbour masks nbr[c * MAXN + u] with class weights w[c].
struct CutView {
    const uint64_t *nbr;
    const int *w;
    int K;
};

// The pass's scalar controls, copied from the parameter space into registers
// once per CTA.
struct PassRegs {
    int n, s, is_low, hmask, load, pre_phase, pre_lambda, write, post, j0, skip_last;
    double amp0;
};

template <typename R>
struct StageCtx {
    typename CT<R>::T *sv0, *sv1;
    const typename CT<R>::T *tab;
    const int *tc;     // this tile's constants [2][16] (function 0 = C, 1 = O)
    const int *ptc;    // this thread's launch constants: ptc[(e * (RB + 1) + i) * NTHR]
    const int *qr;     // [2][2^RB] register-pair terms
    const float *qrf;  // the same as floats
    uint64_t fixed;
    int s, cb, tid;  // high qubit s and contiguous bits cb of this pass's tiles
    bool first;
    R tq;          // t of the rotation: tan beta, or -cot beta when |sin| > |cos|
    R f;           // factor dropped by one butterfly: cos beta or sin beta
    R fn, fn2;     // f^n and f^(2n): one whole layer of butterflies
    R scale0;      // f^j0: butterflies of this layer applied by earlier passes
    R run;         // f^j for the current tile (advanced by every butterfly)
    R amp0;        // 2^(-n/2), the amplitude of the generated |+>^n
    R tq2, f2;     // fused pass: rotation of the second layer
    R run2;        // its f^j (the second layer starts on exact vectors: j = 0)
    bool cot, cot2;  // Ising plans: the layer (second layer) uses the cot form
    // Ising plans: tile values [2][16], tile cost phases [16], per-thread
    // values [2][RB+1][NTHR] and cost phases [RB+1][NTHR], stage terms
    const R *tv;
    const typename CT<R>::T *tp;
    const R *ptv;
    const typename CT<R>::T *ptp;
    const R *qv;                  // [2][32]
    const typename CT<R>::T *qp;  // [32]
};

// ------------------------------------------------ cut values in a stage
// A weighted cut function is quadratic in the bits: flipping vertex u from 0
// to 1 changes it by h_u(x) = sum_c w_c (deg_c(u) - 2 |N_c(u) & x|), and two
// flipped neighbours u, v interact by J_uv = -2 sum_c w_c [uv in E_c]. Write
// a basis state of a tile as x = f | t | r: f the tile's fixed bits, t the
// thread's bits of this stage, r its register bits. Then
//   O(x) = O(f) + sum_{u in t} h_u(f) + sum_{u<v in t} J_uv        (base)
//        + sum_{k in r} (h_k(f) + sum_{u in t} J_ku)             (d_k)
//        + sum_{k<k' in r} J_kk'                                  (Qr[r]).
// O(f) and h_u(f) for the T tile vertices depend on the tile only (the
// producer warp computes them per tile), the t-only sums on the thread only
// (computed once per launch), Qr on the stage only. What is left per thread
// and tile is a subset sum over the 2^RB register states.
template <typename G, int ST, typename V>
__device__ __forceinline__ void cut_terms(const V *tc, const V *pt, int tid, V &base, V (&d)[G::RB])
{
    constexpr int NTB = G::T - G::RB;
    base = tc[15] + pt[0];
#pragma unroll
    for (int j = 0; j < NTB; j++)
        if ((tid >> j) & 1)
            base += tc[G::thr(ST, j)];
#pragma unroll
    for (int k = 0; k < G::RB; k++)
        d[k] = tc[G::reg(ST, k)] + pt[(1 + k) * G::NTHR];
}

// integer cut values (phase-table indices)
template <typename G, int ST>
__device__ __forceinline__ void cut_int(const int *tc, const int *pt, const int *qr, int tid, int (&v)[1 << G::RB])
{
    constexpr int RB = G::RB;
    int base, d[RB];
    cut_terms<G, ST>(tc, pt, tid, base, d);
    v[0] = base;
#pragma unroll
    for (int m = 1; m < (1 << RB); m++) {
        const int top = hibit(m);
        v[m] = v[m ^ (1 << top)] + d[top];
    }
#pragma unroll
    for (int m = 1; m < (1 << RB); m++)
        v[m] += qr[m];
}

// cut values as multipliers of type R (exact: integers below 2^24)
template <typename G, typename R, int ST>
__device__ __forceinline__ void cut_real(const int *tc, const int *pt, const int *qr, const float *qrf, int tid,
                                         R (&v)[1 << G::RB])
{
    constexpr int RB = G::RB;
    int base, d[RB];
    cut_terms<G, ST>(tc, pt, tid, base, d);
    if constexpr (std::is_same<R, float>::value) {
        float df[RB];
#pragma unroll
        for (int k = 0; k < RB; k++)
            df[k] = (float)d[k];
        v[0] = (float)base;
#pragma unroll
        for (int m = 1; m < (1 << RB); m++) {
            const int top = hibit(m);
            v[m] = v[m ^ (1 << top)] + df[top];
        }
#pragma unroll
        for (int m = 1; m < (1 << RB); m++)
            v[m] += qrf[m];
    } else {
        int iv[1 << RB];
        iv[0] = base;
#pragma unroll
        for (int m = 1; m < (1 << RB); m++) {
            const int top = hibit(m);
            iv[m] = iv[m ^ (1 << top)] + d[top];
        }
#pragma unroll
        for (int m = 0; m < (1 << RB); m++)
            v[m] = (R)(iv[m] + qr[m]);
    }
}

// Ising plans: the same quadratic decomposition with real couplings and
// fields. Values O(x) of the thread's 2^RB states from constants rounded
// once to R (tile: tc[15] = O(f), tc[L] = h_L(f); thread: pt; stage: q).
template <typename G, typename R, int ST>
__device__ __forceinline__ void ising_vals(const R *tc, const R *pt, const R *q, int tid, R (&v)[1 << G::RB])
{
    constexpr int RB = G::RB;
    R base, d[RB];
    cut_terms<G, ST, R>(tc, pt, tid, base, d);
    v[0] = base;
#pragma unroll
    for (int m = 1; m < (1 << RB); m++) {
        const int top = hibit(m);
        v[m] = v[m ^ (1 << top)] + d[top];
    }
#pragma unroll
    for (int m = 1; m < (1 << RB); m++)
        v[m] += q[m];
}

// Ising phases P[m] = scale * exp(-i s gamma O(x)) of the thread's states as
// products of unit factors, each computed in FP64 from its exact term and
// rounded once: tp[15] = scale * exp(..O(f)), tp[L] = exp(..h_L(f)) per tile;
// pp[0] (thread-bit pairs), pp[(1 + k) NTHR] (register bit k with the thread
// bits) per thread; qp[m] (register-bit pairs) per stage.
template <typename G, typename C, int ST>
__device__ __forceinline__ void ising_phases(const C *tp, const C *pp, const C *qp, int tid, C (&P)[1 << G::RB])
{
    constexpr int RB = G::RB, NTB = G::T - G::RB;
    C base = cmul(tp[15], pp[0]);
#pragma unroll
    for (int j = 0; j < NTB; j++)
        if ((tid >> j) & 1)
            base = cmul(base, tp[G::thr(ST, j)]);
    C d[RB];
#pragma unroll
    for (int k = 0; k < RB; k++)
        d[k] = cmul(tp[G::reg(ST, k)], pp[(1 + k) * G::NTHR]);
    P[0] = base;
#pragma unroll
    for (int m = 1; m < (1 << RB); m++) {
        const int top = hibit(m);
        P[m] = cmul(P[m ^ (1 << top)], d[top]);
    }
#pragma unroll
    for (int m = 1; m < (1 << RB); m++)
        if (m & (m - 1))
            P[m] = cmul(P[m], qp[m]);
}

// A thread's running sum over its tiles, in FP64 for both precisions: each
// register stage sums its 2^RB products in the amplitude type, and every sum
// across stages, tiles, threads and CTAs is an FP64 add.
template <typename R> struct Acc {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add(R x) { v += (double)x; }
    __device__ __forceinline__ double get() const { return v; }
};

// The butterflies of stage ST due in this pass, with rotation t = tq and
// dropped factor f; run is f^j on entry (j butterflies of the layer already
// applied) and is advanced. Rotations (twisted frame), no rescaling: after j
// butterflies of a layer the vectors carry 1/f^j (restored by the next phase
// table or the last pass), so an inner product taken before butterfly j+1 is
// scaled by f^(2j). In the twisted frame Im<lambda|X_q|phi> sums, over the
// pairs (x, x'), Re(conj(lambda_x') phi_x) - Re(conj(lambda_x) phi_x').
// DUE >= 0: which owned bits are due is fixed at compile time -- all but the
// first DUE owned bits of the stage (the pass shapes the planner makes); DUE
// = -1: decided per bit at run time from A.is_low, A.hmask and cb (any plan).
template <typename G>
__host__ __device__ constexpr int first_owned(int st)
{
    int k = 0;
    while (k < G::RB && !((G::own(st) >> k) & 1))
        k++;
    return k;
}

template <typename R, int NV, int ST, bool COT, int DUE>
__device__ __forceinline__ void mix_regs_form(const PassRegs &A, int cb, R tq, R f, R &run,
                                              typename CT<R>::T (&a)[1 << Geo<R, NV>::RB],
                                              typename CT<R>::T (&l)[1 << Geo<R, NV>::RB], Acc<R> &acc)
{
    using G = Geo<R, NV>;
    using C = typename CT<R>::T;
    constexpr int RB = G::RB, NR = 1 << RB;
    R gb = 0, sc = run;
#pragma unroll
    for (int k = 0; k < RB; k++) {
        if (!((G::own(ST) >> k) & 1))
            continue;
        bool due = true;
        if constexpr (DUE >= 0)
            due = k >= first_owned<G>(ST) + DUE;
        else if (G::reg(ST, k) >= cb)
            due = (A.hmask >> (G::reg(ST, k) - cb)) & 1;
        else
            due = A.is_low;
        if (!due)
            continue;
        C ipp[2], ipn[2];
        ipp[0] = ipp[1] = ipn[0] = ipn[1] = mkc<C>((R)0, (R)0);
#pragma unroll
        for (int m = 0; m < NR; m++) {
            if (m & (1 << k))
                continue;
            const int m1 = m | (1 << k);
            if constexpr (NV == 2) {
                const int c = (m >> (k == 0 ? 1 : 0)) & 1;
                dot_acc(ipp[c], l[m1], a[m]);
                dot_acc(ipn[c], l[m], a[m1]);
                if constexpr (COT)
                    rotc(l[m], l[m1], tq);
                else
                    rot(l[m], l[m1], tq);
            }
            if constexpr (COT)
                rotc(a[m], a[m1], tq);
            else
                rot(a[m], a[m1], tq);
        }
        if constexpr (NV == 2) {
            const R q = ((ipp[0].x + ipp[0].y) + (ipp[1].x + ipp[1].y)) - ((ipn[0].x + ipn[0].y) + (ipn[1].x + ipn[1].y));
            gb = fma(q, sc * sc, gb);
        }
        sc *= f;
    }
    run = sc;
    if constexpr (NV == 2)
        acc.add(gb);
}

// cot (Ising plans only, decided per layer) selects the butterfly form once
// for the whole stage, outside the unrolled loops
template <typename R, int NV, int ST, bool IS = false, int DUE = -1>
__device__ __forceinline__ void mix_regs(const PassRegs &A, int cb, R tq, R f, R &run,
                                         typename CT<R>::T (&a)[1 << Geo<R, NV>::RB],
                                         typename CT<R>::T (&l)[1 << Geo<R, NV>::RB], Acc<R> &acc,
                                         bool cot = false)
{
    if (IS && cot)
        mix_regs_form<R, NV, ST, true, DUE>(A, cb, tq, f, run, a, l, acc);
    else
        mix_regs_form<R, NV, ST, false, DUE>(A, cb, tq, f, run, a, l, acc);
}

// One register stage of a pass over the tile(s) in sv0 (and sv1 for NV = 2).
// FUSE (last stage of a fused pass): after this layer's operations the second
// layer's butterflies of the same stage follow, their dE/dbeta into acc2.
// IS: an Ising plan (real values, phases as products of unit factors, cot form
// of the rotation where the layer needs it).
template <typename R, int NV, int ST, bool OPS, bool FUSE = false, bool IS = false, int DUE = -1>
__device__ __forceinline__ void run_stage(const PassRegs &A, StageCtx<R> &X,
                                          typename CT<R>::T (&a)[1 << Geo<R, NV>::RB],
                                          typename CT<R>::T (&l)[1 << Geo<R, NV>::RB], Acc<R> &acc0,
                                          Acc<R> &acc1, Acc<R> &acc2)
{
    using G = Geo<R, NV>;
    using C = typename CT<R>::T;
    constexpr int RB = G::RB, NR = 1 << RB, NTB = G::T - RB;
    constexpr bool LAST = (ST == G::NST - 1);

    const uint32_t base = stage_base<G, ST>((uint32_t)X.tid);
    const uint32_t sb = G::swz(base);

    if (ST == 0 && !A.load) {  // |+>^n in the twisted frame: 2^(-n/2) i^|x|
        // the four values amp * i^((c0 + j) & 3) once, then a compile-time
        // choice by the register index's own bit count
        const int c0 = (__popcll(X.fixed) + __popc(base)) & 3;
        const R amp = X.amp0;
        C zc[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int e = (c0 + j) & 3;
            zc[j] = mkc<C>(e == 0 ? amp : e == 2 ? -amp : (R)0, e == 1 ? amp : e == 3 ? -amp : (R)0);
        }
#pragma unroll
        for (int m = 0; m < NR; m++)
            a[m] = zc[__popc(m) & 3];
    } else {
        load_regs<R, NV, ST>(X.sv0, sb, a);
        if constexpr (NV == 2)
            if (!(OPS && X.first && A.pre_lambda))
                load_regs<R, NV, ST>(X.sv1, sb, l);
    }

    // cut-function constants: function 0 is C (cost), 1 the observable O
    const int *tc0 = X.tc, *tc1 = X.tc + 16;
    const int *pt0 = X.ptc + X.tid, *pt1 = X.ptc + (RB + 1) * G::NTHR + X.tid;
    // the values O_e(x) of the thread's states (real; exact integers for cut functions)
    auto values = [&](int e, R (&v)[NR]) {
        if constexpr (IS)
            ising_vals<G, R, ST>(X.tv + 16 * e, X.ptv + e * (RB + 1) * G::NTHR + X.tid, X.qv + 32 * e, X.tid, v);
        else
            cut_real<G, R, ST>(e ? tc1 : tc0, e ? pt1 : pt0, X.qr + 32 * e, X.qrf + 32 * e, X.tid, v);
    };
    // the cost layer's phase factors of the thread's states (this pass's table)
    auto phases = [&](C (&P)[NR]) {
        if constexpr (IS) {
            ising_phases<G, C, ST>(X.tp, X.ptp + X.tid, X.qp, X.tid, P);
        } else {
            int cv[NR];
            cut_int<G, ST>(tc0, pt0, X.qr, X.tid, cv);
#pragma unroll
            for (int m = 0; m < NR; m++)
                P[m] = X.tab[cv[m]];
        }
    };

    if (OPS && ST == 0 && A.pre_phase) {
        C P[NR];
        phases(P);
#pragma unroll
        for (int m = 0; m < NR; m++)
            a[m] = cmul(a[m], P[m]);
    }
    if constexpr (NV == 2) {
        if (OPS && X.first && A.pre_lambda) {  // lambda = O phi, from the stored final state
            R ov[NR];
            values(1, ov);
#pragma unroll
            for (int m = 0; m < NR; m++)
                l[m] = mkc<C>(a[m].x * ov[m], a[m].y * ov[m]);
        }
    }

    mix_regs<R, NV, ST, IS, DUE>(A, X.cb, X.tq, X.f, X.run, a, l, acc0, X.cot);

    if (OPS && LAST && (A.post & POST_RESCALE)) {  // the stored state is the exact one
#pragma unroll
        for (int m = 0; m < NR; m++) {
            a[m].x *= X.fn;
            a[m].y *= X.fn;
        }
    }

    if (OPS && LAST && (A.post & POST_REDUCE)) {
        R ov[NR];
        values(1, ov);
        R e = 0;
#pragma unroll
        for (int m = 0; m < NR; m++)
            e += (a[m].x * a[m].x + a[m].y * a[m].y) * ov[m];
        acc0.add((A.post & POST_RESCALE) ? e : e * X.fn2);
    }
    if constexpr (NV == 2) {
        if (OPS && LAST && (A.post & (POST_GAMMA | POST_PHASE_CONJ))) {
            if (A.post & POST_GAMMA) {
                R cr[NR];
                values(0, cr);
                R g = 0;
#pragma unroll
                for (int m = 0; m < NR; m++)
                    g += cr[m] * im_conj_mul(l[m], a[m]);
                acc1.add(g * X.fn2);  // both vectors carry 1/f^n here
            }
            if (A.post & POST_PHASE_CONJ) {  // inverse cost layer, restoring f^n
                C P[NR];
                phases(P);
#pragma unroll
                for (int m = 0; m < NR; m++) {
                    a[m] = cmul(a[m], P[m]);
                    l[m] = cmul(l[m], P[m]);
                }
            }
        }
    }
    if constexpr (NV == 1) {
        if (OPS && LAST && (A.post & POST_PHASE)) {  // the next layer's cost phase
            C P[NR];
            phases(P);
#pragma unroll
            for (int m = 0; m < NR; m++)
                a[m] = cmul(a[m], P[m]);
        }
    }
    if constexpr (FUSE && LAST)
        mix_regs<R, NV, ST, IS, DUE>(A, X.cb, X.tq2, X.f2, X.run2, a, l, acc2, X.cot2);
    if (!LAST || A.write) {
        store_regs<R, NV, ST>(X.sv0, sb, a);
        if constexpr (NV == 2)
            store_regs<R, NV, ST>(X.sv1, sb, l);
    }
}

// A stage of the second layer of a fused pass: load, its butterflies, store.
template <typename R, int NV, int ST, bool IS = false, int DUE = -1>
__device__ __forceinline__ void mix_stage(const PassRegs &A, StageCtx<R> &X,
                                          typename CT<R>::T (&a)[1 << Geo<R, NV>::RB],
                                          typename CT<R>::T (&l)[1 << Geo<R, NV>::RB], Acc<R> &acc2)
{
    using G = Geo<R, NV>;
    const uint32_t base = stage_base<G, ST>((uint32_t)X.tid);
    const uint32_t sb = G::swz(base);
    load_regs<R, NV, ST>(X.sv0, sb, a);
    if constexpr (NV == 2)
        load_regs<R, NV, ST>(X.sv1, sb, l);
    mix_regs<R, NV, ST, IS, DUE>(A, X.cb, X.tq2, X.f2, X.run2, a, l, acc2, X.cot2);
    store_regs<R, NV, ST>(X.sv0, sb, a);
    if constexpr (NV == 2)
        store_regs<R, NV, ST>(X.sv1, sb, l);
}

// Which owned bits of stage st a pass with this shape transforms: 0 every
// owned bit, 1 all but the first, -1 another set. A high pass transforms the
// tile bits from cb up, a low pass those below cb plus the high bits in hmask.
template <typename G>
__host__ __device__ inline int due_form(int st, int is_low, int hmask, int cb)
{
    uint32_t own = 0, due = 0;
    for (int k = 0; k < G::RB; k++) {
        if (!((G::own(st) >> k) & 1))
            continue;
        own |= 1u << k;
        const int bit = G::reg(st, k);
        if (bit >= cb ? ((hmask >> (bit - cb)) & 1) : is_low)
            due |= 1u << k;
    }
    return due == own ? 0 : due == (own & (own - 1u)) ? 1 : -1;
}

// A register stage in the compiled form of its due pattern d (complex64: the
// run-time checks cost about a third of a stage's time; complex128 passes are
// bound by FP64 arithmetic and keep the checks).
template <typename R, int NV, int ST, bool OPS, bool FUSE, bool IS>
__device__ __forceinline__ void run_stage_due(int d, const PassRegs &A, StageCtx<R> &X,
                                              typename CT<R>::T (&a)[1 << Geo<R, NV>::RB],
                                              typename CT<R>::T (&l)[1 << Geo<R, NV>::RB], Acc<R> &acc0,
                                              Acc<R> &acc1, Acc<R> &acc2)
{
    if constexpr (std::is_same<R, float>::value) {
        if (d == 0)
            return run_stage<R, NV, ST, OPS, FUSE, IS, 0>(A, X, a, l, acc0, acc1, acc2);
        if (d == 1)
            return run_stage<R, NV, ST, OPS, FUSE, IS, 1>(A, X, a, l, acc0, acc1, acc2);
    }
    run_stage<R, NV, ST, OPS, FUSE, IS, -1>(A, X, a, l, acc0, acc1, acc2);
}

template <typename R, int NV, int ST, bool IS>
__device__ __forceinline__ void mix_stage_due(int d, const PassRegs &A, StageCtx<R> &X,
                                              typename CT<R>::T (&a)[1 << Geo<R, NV>::RB],
                                              typename CT<R>::T (&l)[1 << Geo<R, NV>::RB], Acc<R> &acc2)
{
    if constexpr (std::is_same<R, float>::value) {
        if (d == 0)
            return mix_stage<R, NV, ST, IS, 0>(A, X, a, l, acc2);
        if (d == 1)
            return mix_stage<R, NV, ST, IS, 1>(A, X, a, l, acc2);
    }
    mix_stage<R, NV, ST, IS, -1>(A, X, a, l, acc2);
}

// Named barrier 1 spans the NTHR compute threads only (the producer warp
// never takes part).
template <int NTHR>
__device__ __forceinline__ void compute_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(NTHR) : "memory");
}

// Barrier over the compute threads that also returns, to every thread, the OR
// of a per-thread flag: a decision all threads take alike.
template <int NTHR>
__device__ __forceinline__ bool compute_sync_or(bool flag)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred ip, op;\n\t"
        "setp.ne.u32 ip, %1, 0;\n\t"
        "barrier.cta.red.or.pred op, 1, %2, ip;\n\t"
        "selp.u32 %0, 1, 0, op;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)flag), "n"(NTHR)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Tiles of CTA c: interleaved (c, c+G, c+2G, ...) when chunk == 0, else the
// contiguous range [c*chunk, (c+1)*chunk) -- used for batches so that a CTA
// meets each parameter point once.
__device__ __forceinline__ unsigned cta_tile(unsigned c, unsigned k, unsigned grid, unsigned chunk)
{
    return chunk ? c * chunk + k : c + k * grid;
}

__device__ __forceinline__ unsigned cta_tile_count(unsigned c, unsigned grid, unsigned chunk, unsigned total)
{
    if (chunk) {
        const unsigned lo = c * chunk;
        return lo < total ? (total - lo < chunk ? total - lo : chunk) : 0;
    }
    return c < total ? (total - c + grid - 1) / grid : 0;
}

// Was any tile of point b processed by CTA c?
__device__ __forceinline__ bool cta_touches(unsigned c, unsigned b, unsigned tiles, unsigned grid, unsigned total,
                                            unsigned chunk)
{
    const unsigned lo = b * tiles, hi = lo + tiles;
    if (chunk) {
        const unsigned c0 = c * chunk, c1 = c0 + cta_tile_count(c, grid, chunk, total);
        return c0 < hi && lo < c1;
    }
    unsigned g0 = c;
    if (g0 < lo)
        g0 += ((lo - c + grid - 1) / grid) * grid;
    return g0 < hi && g0 < total;
}

// partials[slot][b][cta]; the last CTA to finish sums them in a fixed order:
// one warp per (slot, point), lanes over the CTAs, then a fixed shuffle tree
__device__ void pass_final_reduce(const PassArgs &A, unsigned total)
{
    __shared__ unsigned s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(A.counter, 1u) == gridDim.x - 1u) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    const unsigned G = gridDim.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int job = w; job < 3 * A.B; job += nw) {
        const int slot = job / A.B, b = job - slot * A.B;
        if (A.slot_idx[slot] < 0)
            continue;
        const double *src = A.partials + ((size_t)slot * A.B + b) * G;
        double a = 0.0;
        for (unsigned c = lane; c < G; c += 32)
            if (cta_touches(c, (unsigned)b, (unsigned)A.tiles, G, total, (unsigned)A.chunk))
                a += __ldcg(src + c);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0)
            A.out[(size_t)b * A.out_stride + A.slot_idx[slot]] += A.slot_scale[slot] * a;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        *A.counter = 0u;
}

// A pass's operation flags as one word: load, pre_phase, pre_lambda and
// write in bits 0-3, the PostOp bits from bit 4. The complex64 kernels run the
// flag words of the planner's usual passes in a compute loop compiled for
// them (branches and the code of operations not taken leave the per-tile
// path); any other word runs the loop that reads the flags at run time.
__host__ __device__ constexpr int flag_word(int load, int pre_phase, int pre_lambda, int write, int post)
{
    return (load ? 1 : 0) | (pre_phase ? 2 : 0) | (pre_lambda ? 4 : 0) | (write ? 8 : 0) | (post << 4);
}
constexpr int FW_FWD_FIRST = flag_word(0, 1, 0, 1, 0);                          // |+> generated, first phase
constexpr int FW_FWD_LAST = flag_word(1, 0, 0, 1, POST_REDUCE | POST_RESCALE);  // energy, state kept
constexpr int FW_FWD_ENERGY = flag_word(1, 0, 0, 0, POST_REDUCE);               // energy only
constexpr int FW_FWD_FUSED = flag_word(1, 0, 0, 1, POST_PHASE);
constexpr int FW_ADJ_FIRST = flag_word(1, 0, 1, 1, 0);                          // lambda = O phi
constexpr int FW_ADJ_LAST = flag_word(1, 0, 0, 0, POST_GAMMA);                  // layer 0 ends
constexpr int FW_ADJ_BOUNDARY = flag_word(1, 0, 0, 1, POST_GAMMA | POST_PHASE_CONJ);

// Persistent tiled pass over A.B statevectors, warp-specialised. CTA c takes
// tiles c, c+G, c+2G, ... (G = gridDim.x) of the B x tiles sequence. The last
// warp is the producer: its lane 0 keeps NSTAGE tiles in flight (TMA loads)
// and writes finished tiles back (TMA stores). The NTHR compute threads run
// the register stages. Per stage buffer s two mbarriers hand the buffer over:
// full[s] (producer -> compute: tile loaded, or buffer free in a generating
// pass) and done[s] (compute -> producer: results in shared memory).
// MODE 0: mixer only; 1: with cut-function work on one graph; 2: the same
// with point b of the batch being its own graph (A.pt[b]); 3: as 1, and the
// pass is fused (A.fuse): after the last stage's operations the mixer of
// layer A.layer2 is applied to the same qubits, last stage first. Ising
// plans: 4 (as 1), 5 (as 3), 6 (as 0), with real-valued cut functions, phase
// factors built from products and the cot form where a layer needs it.
template <typename R, int NV, int MODE>
__global__ void __maxnreg__((Geo<R, NV>::MAXREG))
    k_pass(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1,
           const __grid_constant__ PassArgs A)
{
    constexpr bool OPS = MODE != 0 && MODE != 6, MG = MODE == 2, FUSE = MODE == 3 || MODE == 5, IS = MODE >= 4;
    using G = Geo<R, NV>;
    using C = typename CT<R>::T;
    constexpr int NR = 1 << G::RB, NS = G::NSTAGE, NTHR = G::NTHR;
    constexpr uint32_t TB = (uint32_t)tile_bytes<R, NV>();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment (TMA 128-byte swizzle) by pointer arithmetic on the
    // shared array itself, so every tile access stays a shared-memory access
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[NS], done[NS];
    __shared__ double pred[2][3][32];  // per-warp sums of a finished point, two buffers
    __shared__ int s_flag;
    __shared__ int obs_w[MAXK], cost_w[MAXK];
    __shared__ int tcs[IS ? 1 : NS][2][16];              // per buffer: O(f) and h_u(f) of its tile
    __shared__ int ptc[IS ? 1 : 2 * (G::RB + 1) * NTHR];  // per thread: t-only terms of each function
    __shared__ int qr[2][2][32];                         // [slot][function]: register-pair terms
    __shared__ float qrf[2][2][32];
    // Ising plans: tile values and cost phases per buffer, stage terms (the
    // per-thread terms live in the dynamic region after the tiles)
    __shared__ R tvs[IS ? NS : 1][2][16];
    __shared__ C tps[IS ? NS : 1][16];
    __shared__ R qvs[IS ? 2 : 1][32];
    __shared__ C qps[IS ? 2 : 1][32];
    __shared__ double isd[IS ? 2 : 1][IS ? MAXN : 1];  // d_u = h_u + sum_v W_uv of both functions

    const int tid = threadIdx.x;
    C *tab = reinterpret_cast<C *>(sm + (size_t)NS * NV * TB);
    uint64_t *cost_nbr = reinterpret_cast<uint64_t *>(tab + 2 * MAXTAB);  // two table slots
    uint64_t *obs_nbr = cost_nbr + MAXK * MAXN;
    // Ising plans reuse that region: per-thread values [2][RB+1][NTHR] and cost phases [RB+1][NTHR]
    R *ptv = reinterpret_cast<R *>(sm + (size_t)NS * NV * TB);
    C *ptp = reinterpret_cast<C *>(ptv + 2 * (G::RB + 1) * NTHR);

    const unsigned total = (unsigned)A.tiles * (unsigned)A.B;
    const unsigned grid = gridDim.x;
    const unsigned niter = cta_tile_count(blockIdx.x, grid, (unsigned)A.chunk, total);
    // tile = 2^cb contiguous amplitudes x 2^(T-cb) rows along qubits s..
    const int cb = A.cb, hb = G::T - A.cb;
    const int midbits = A.s - cb;
    const unsigned tiles_per_hi = (unsigned)A.tiles >> midbits;  // 2^(n - s - hb)
    const bool reduce = A.slot_idx[0] >= 0 || A.slot_idx[1] >= 0 || A.slot_idx[2] >= 0;

    if (tid == 0) {
        s_flag = *reinterpret_cast<volatile int *>(A.err) ? 1 : 0;
        for (int s = 0; s < NS; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&done[s], NTHR);
        }
        fence_barrier_init();
    }
    if constexpr (!IS) {
        for (int i = tid; i < A.cost.K * MAXN; i += blockDim.x)
            cost_nbr[i] = A.cost.nbr[i / MAXN][i % MAXN];
        for (int i = tid; i < A.obs.K * MAXN; i += blockDim.x)
            obs_nbr[i] = A.obs.nbr[i / MAXN][i % MAXN];
        if (tid < MAXK) {
            obs_w[tid] = A.obs.w[tid];
            cost_w[tid] = A.cost.w[tid];
        }
    }
    __syncthreads();
    if (s_flag)
        return;

    // The register stage that evaluates each cut function in this pass, or -1:
    // C for the phase of a forward low pass (stage 0), for the next layer's
    // phase in a fused forward pass and for the gradient and inverse phase of
    // the last adjoint pass of a layer (last stage); O for
    // lambda = O phi (first stage of the first adjoint pass) and for the
    // energy (last stage of the last forward pass).
    int est[2] = {-1, -1};
    if (OPS) {
        if (A.pre_phase)
            est[0] = 0;
        else if (NV == 2 && (A.post & (POST_GAMMA | POST_PHASE_CONJ)))
            est[0] = G::NST - 1;
        else if (NV == 1 && (A.post & POST_PHASE))
            est[0] = G::NST - 1;
        if (NV == 2 && A.pre_lambda)
            est[1] = A.is_low ? 0 : 1;
        else if (A.post & POST_REDUCE)
            est[1] = G::NST - 1;
    }
    // vertex of local tile bit L; for a batch of graphs (MG) the two cut
    // functions of point b, read from the batch's global array (a single
    // graph uses the shared-memory copies above directly)
    auto gq = [&](int L) { return L < A.cb ? L : A.s + L - A.cb; };
    auto views = [&](unsigned b, CutView (&v)[2]) {
        const GraphFns &gf = A.pt[b];
        v[0] = CutView{&gf.cost.nbr[0][0], gf.cost.w, gf.cost.K};
        v[1] = CutView{&gf.obs[A.pt_obs].nbr[0][0], gf.obs[A.pt_obs].w, gf.obs[A.pt_obs].K};
    };
    CutView curv[2];  // per-point graphs: the current point's functions
    auto wgt = [&](int e, int u, int v) -> int {
        int w = 0;
        if constexpr (MG) {
            const CutView &f = curv[e];
            for (int c = 0; c < f.K; c++)
                w += f.w[c] * (int)((f.nbr[c * MAXN + u] >> v) & 1ull);
        } else {  // the shared-memory copies of the launch's one graph
            const uint64_t *nb = e == 0 ? cost_nbr : obs_nbr;
            const int *ww = e == 0 ? cost_w : obs_w;
            const int K = e == 0 ? A.cost.K : A.obs.K;
            for (int c = 0; c < K; c++)
                w += ww[c] * (int)((nb[c * MAXN + u] >> v) & 1ull);
        }
        return w;
    };
    // launch constants of the quadratic decomposition, into qr slot `qs`
    // (each thread writes its own ptc entries)
    auto launch_consts = [&](int qs) {
        constexpr int RB = G::RB, NTB = G::T - G::RB;
#pragma unroll
        for (int e = 0; e < 2; e++) {
            const int st = est[e];
            if (st < 0)
                continue;
            int q = 0;
            for (int j = 0; j < NTB; j++)
                for (int j2 = 0; j2 < j; j2++)
                    if (((tid >> j) & 1) && ((tid >> j2) & 1))
                        q -= 2 * wgt(e, gq(G::thr(st, j)), gq(G::thr(st, j2)));
            ptc[(e * (RB + 1)) * NTHR + tid] = q;
            for (int kk = 0; kk < RB; kk++) {
                int dk = 0;
                for (int j = 0; j < NTB; j++)
                    if ((tid >> j) & 1)
                        dk -= 2 * wgt(e, gq(G::reg(st, kk)), gq(G::thr(st, j)));
                ptc[(e * (RB + 1) + 1 + kk) * NTHR + tid] = dk;
            }
            if (tid < (1 << RB)) {
                int qq = 0;
                for (int kk = 0; kk < RB; kk++)
                    for (int k2 = 0; k2 < kk; k2++)
                        if (((tid >> kk) & 1) && ((tid >> k2) & 1))
                            qq -= 2 * wgt(e, gq(G::reg(st, kk)), gq(G::reg(st, k2)));
                qr[qs][e][tid] = qq;
                qrf[qs][e][tid] = (float)qq;
            }
        }
    };
    // Ising plans: the real couplings of function e between vertices u and v
    auto ising_fn = [&](int e) -> const IsingFn * { return e == 0 ? A.icost : A.iobs; };
    // this thread's terms of function e in stage st, in FP64: thread-bit
    // pairs (q), register bit k with the thread bits (dk), and for tid < 2^RB
    // the register-bit pairs of subset tid (qq)
    auto ising_terms = [&](int e, int st, double &q, double (&dk)[G::RB], double &qq) {
        constexpr int RB = G::RB, NTB = G::T - G::RB;
        const IsingFn *F = ising_fn(e);
        q = 0.0;
        for (int j = 0; j < NTB; j++)
            for (int j2 = 0; j2 < j; j2++)
                if (((tid >> j) & 1) && ((tid >> j2) & 1))
                    q -= 2.0 * F->W[gq(G::thr(st, j))][gq(G::thr(st, j2))];
        for (int kk = 0; kk < RB; kk++) {
            dk[kk] = 0.0;
            for (int j = 0; j < NTB; j++)
                if ((tid >> j) & 1)
                    dk[kk] -= 2.0 * F->W[gq(G::reg(st, kk))][gq(G::thr(st, j))];
        }
        qq = 0.0;
        if (tid < (1 << RB))
            for (int kk = 0; kk < RB; kk++)
                for (int k2 = 0; k2 < kk; k2++)
                    if (((tid >> kk) & 1) && ((tid >> k2) & 1))
                        qq -= 2.0 * F->W[gq(G::reg(st, kk))][gq(G::reg(st, k2))];
    };
    // the cost layer's phase angle per unit of the cost function for point b:
    // -gamma forward (exp(-i gamma C)), +gamma for the inverse layer
    auto ising_angle = [&](unsigned b) { return -A.sign_s * A.gam[(size_t)b * A.p + A.tab_layer]; };
    const bool cost_phase = A.pre_phase || (A.post & (POST_PHASE | POST_PHASE_CONJ));
    if constexpr (IS) {
        // flip costs from the all-zero state, for the producer's tile constants
        if (tid < 2 * MAXN) {
            const int e = tid / MAXN, u = tid % MAXN;
            if (est[e] >= 0 && u < A.n) {
                const IsingFn *F = ising_fn(e);
                double d = F->h[u];
                for (int v = 0; v < A.n; v++)
                    d += F->W[u][v];
                isd[e][u] = d;
            }
        }
        __syncthreads();
        if (tid < NTHR) {
            for (int e = 0; e < 2; e++) {
                if (est[e] < 0)
                    continue;
                double q, dk[G::RB], qq;
                ising_terms(e, est[e], q, dk, qq);
                ptv[(e * (G::RB + 1)) * NTHR + tid] = (R)q;
                for (int kk = 0; kk < G::RB; kk++)
                    ptv[(e * (G::RB + 1) + 1 + kk) * NTHR + tid] = (R)dk[kk];
                if (tid < (1 << G::RB))
                    qvs[e][tid] = (R)qq;
            }
        }
    } else if (tid < NTHR && !MG && (est[0] >= 0 || est[1] >= 0)) {
        launch_consts(0);
    }

    const int tiles_log2 = __ffs(A.tiles) - 1;  // tiles per state: a power of two
    auto tile_coords = [&](unsigned k, unsigned &b, unsigned &t, unsigned &mid, int &c4) {
        const unsigned g = cta_tile(blockIdx.x, k, grid, (unsigned)A.chunk);
        b = g >> tiles_log2;
        t = g & ((unsigned)A.tiles - 1u);
        mid = t & ((1u << midbits) - 1u);
        const unsigned hi = t >> midbits;
        c4 = (int)(hi + b * tiles_per_hi);
    };

    if (tid >= NTHR) {
        // ------------------------------------------------------ producer
        // Lane 0 issues the TMA copies and waits on the mbarriers; the whole
        // warp computes each tile's cut constants O(f), h_u(f) before the
        // tile's buffer is handed over (the arrive on full[s] releases them).
        const int lane = tid - NTHR;
        // Ising plans: O(f) and h_L(f) in FP64, rounded once to R, and for the
        // cost the unit phase factors of this tile's point (O(f)'s carrying
        // the table's scale f^n). With g_u(f) = sum_{v in f} W_uv and
        // d_u = h_u + sum_v W_uv (the flip cost of u from an all-zero state):
        //   O(f) = sum_{u in f} (d_u - g_u(f)),   h_u(f) = d_u - 2 g_u(f),
        // since [f_u != f_v] = f_u + f_v - 2 f_u f_v. Lanes take vertices;
        // every lane loops over the same set bits of f.
        auto tile_consts_ising = [&](unsigned k, int s) {
            unsigned b, t, mid;
            int c4;
            tile_coords(k, b, t, mid, c4);
            const uint64_t f = ((uint64_t)mid << cb) | ((uint64_t)(t >> midbits) << (A.s + hb));
            for (int e = 0; e < 2; e++) {
                if (est[e] < 0)
                    continue;
                const IsingFn *F = ising_fn(e);
                double os = 0.0, hl[2] = {0.0, 0.0};  // lane's vertices u = lane, lane + 32
                for (int j = 0; j < 2; j++) {
                    const int u = lane + 32 * j;
                    if (u >= A.n)
                        continue;
                    double g = 0.0;
                    const double d = isd[e][u];
                    for (uint64_t rest = f; rest; rest &= rest - 1)
                        g += F->W[u][__ffsll((long long)rest) - 1];
                    if ((f >> u) & 1ull)
                        os += d - g;
                    hl[j] = d - 2.0 * g;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    os += __shfl_xor_sync(0xffffffffu, os, o);
                // h_L(f) of local bit L (vertex gq(L)) from the lane holding that vertex
                double hs = 0.0;
                {
                    const int u = lane < G::T ? gq(lane) : 0;
                    const double h0 = __shfl_sync(0xffffffffu, hl[0], u & 31);
                    const double h1 = __shfl_sync(0xffffffffu, hl[1], u & 31);
                    hs = u < 32 ? h0 : h1;
                }
                if (lane < G::T)
                    tvs[s][e][lane] = (R)hs;
                if (lane == 0)
                    tvs[s][e][15] = (R)os;
                if (e == 0 && cost_phase) {
                    const double ang = ising_angle(b);
                    if (lane < G::T)
                        tps[s][lane] = unit_phase<R>(ang * hs);
                    if (lane == 0) {
                        const C sc = reinterpret_cast<const C *>(A.tab)[(size_t)b * A.p + A.tab_layer];
                        C z = unit_phase<R>(ang * os);
                        z.x *= sc.x;
                        z.y *= sc.x;
                        tps[s][15] = z;
                    }
                }
            }
        };
        auto tile_consts = [&](unsigned k, int s) {
            if (est[0] < 0 && est[1] < 0)
                return;
            if constexpr (IS) {
                tile_consts_ising(k, s);
                return;
            }
            unsigned b, t, mid;
            int c4;
            tile_coords(k, b, t, mid, c4);
            const uint64_t f = ((uint64_t)mid << cb) | ((uint64_t)(t >> midbits) << (A.s + hb));
            CutView v[2];
            if constexpr (MG)
                views(b, v);
#pragma unroll
            for (int e = 0; e < 2; e++) {
                if (est[e] < 0)
                    continue;
                const int K = MG ? v[e].K : (e == 0 ? A.cost.K : A.obs.K);
                int hs = 0, os = 0;
                for (int c = 0; c < K; c++) {
                    const uint64_t *nb = MG ? v[e].nbr + c * MAXN : (e == 0 ? cost_nbr : obs_nbr) + c * MAXN;
                    const int w = MG ? v[e].w[c] : (e == 0 ? cost_w[c] : obs_w[c]);
                    if (lane < G::T) {
                        const uint64_t m = nb[gq(lane)];
                        hs += w * (__popcll(m) - 2 * __popcll(m & f));
                    }
                    for (int u = lane; u < A.n; u += 32)
                        if ((f >> u) & 1ull)
                            os += w * __popcll(nb[u] & ~f);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    os += __shfl_xor_sync(0xffffffffu, os, o);
                if (lane < G::T)
                    tcs[s][e][lane] = hs;
                if (lane == 0)
                    tcs[s][e][15] = os;
            }
        };
        bool ok = true;
        long long last_fill[NS];  // newest tile loaded into each buffer (lane 0)
        for (int s = 0; s < NS; s++)
            last_fill[s] = -1;
        auto fill = [&](unsigned k) {  // tile k into buffer k % NS
            const int s = (int)(k % NS);
            tile_consts(k, s);
            __syncwarp();
            if (lane != 0)
                return;
            if (A.drop_first_load && k == 0 && blockIdx.x == 0)
                return;  // test hook: this tile's load is never issued, its wait runs out
            last_fill[s] = (long long)k;
            if (A.load) {
                unsigned b, t, mid;
                int c4;
                tile_coords(k, b, t, mid, c4);
                unsigned char *buf = sm + (size_t)s * NV * TB;
                const int c1 = A.wide_rows ? 0 : (int)mid, c2 = A.wide_rows ? (int)mid : 0;
                mbar_arrive_expect_tx(&full[s], (uint32_t)A.nvec_io * TB);
                tma_load_5d(buf, &map0, &full[s], 0, c1, c2, 0, c4);
                if (A.nvec_io == 2)
                    tma_load_5d(buf + TB, &map1, &full[s], 0, c1, c2, 0, c4);
            } else {
                mbar_arrive(&full[s]);  // generating pass: the buffer is free
            }
        };
        for (unsigned k = 0; k < (unsigned)NS && k < niter; k++)
            fill(k);
        for (unsigned k = 0; k < niter && ok; k++) {
            const int s = (int)(k % NS);
            int good = 1;
            if (lane == 0) {
                good = mbar_wait_bounded(&done[s], (k / NS) & 1u) && !*reinterpret_cast<volatile int *>(&s_flag);
                if (good && A.write) {
                    unsigned b, t, mid;
                    int c4;
                    tile_coords(k, b, t, mid, c4);
                    unsigned char *buf = sm + (size_t)s * NV * TB;
                    const int c1 = A.wide_rows ? 0 : (int)mid, c2 = A.wide_rows ? (int)mid : 0;
                    tma_store_5d(&map0, buf, 0, c1, c2, 0, c4);
                    if (NV == 2)
                        tma_store_5d(&map1, buf + TB, 0, c1, c2, 0, c4);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    if (k + NS < niter)  // the buffer is reloaded: its store must have read it
                        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                }
            }
            good = __shfl_sync(0xffffffffu, good, 0);
            if (!good) {
                ok = false;
                break;
            }
            if (k + NS < niter)
                fill(k + NS);
        }
        if (lane == 0) {
            if (!ok) {
                atomicExch(A.err, 1);
                s_flag = 1;
                if (A.load)  // no TMA load may still be writing shared memory at exit
                    for (int s = 0; s < NS; s++)
                        if (last_fill[s] >= 0)
                            mbar_wait_bounded(&full[s], (unsigned)((last_fill[s] / NS) & 1));
            }
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        }
    } else {
        // ------------------------------------------------------- compute
        // FL: the flag word this loop is compiled for, or -1 (read from A)
        auto compute = [&](auto flc) {
        constexpr int FL = decltype(flc)::value;
        const PassRegs P{A.n, A.s, A.is_low, A.hmask,
                         FL < 0 ? A.load : (FL & 1),
                         FL < 0 ? A.pre_phase : (FL >> 1) & 1,
                         FL < 0 ? A.pre_lambda : (FL >> 2) & 1,
                         FL < 0 ? A.write : (FL >> 3) & 1,
                         FL < 0 ? A.post : FL >> 4,
                         A.j0, A.skip_last, A.amp0};
        Acc<R> acc0, acc1, acc2;
        acc0.zero();
        acc1.zero();
        acc2.zero();
        int cur_b = -1;
        StageCtx<R> X;
        X.tab = tab;
        X.ptc = ptc;
        X.qr = &qr[0][0][0];
        X.qrf = &qrf[0][0][0];
        X.ptv = ptv;
        X.ptp = ptp;
        X.qv = &qvs[0][0];
        X.qp = &qps[0][0];
        X.cot = X.cot2 = false;
        X.s = A.s;
        X.cb = cb;
        X.tid = tid;
        X.amp0 = (R)A.amp0;
        X.first = true;

        // A point change costs no extra barrier. The phase table has two
        // slots (the one being replaced was last read before the previous
        // barrier), and the finished point's sums are warp-reduced into
        // pred[parity] and written out by thread 0 after the next barrier.
        // pred alternates between two buffers, so a warp that stashes the
        // following point cannot overwrite sums thread 0 has not read yet:
        // that stash comes after a barrier thread 0 only reaches when done.
        const int lane = tid & 31, warp = tid >> 5;
        int pend_b = -1, tslot = 1, par = 1;
        auto stash = [&](int b) {
            double s0 = acc0.get(), s1 = acc1.get(), s2 = acc2.get();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                if constexpr (FUSE)
                    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            }
            par ^= 1;
            if (lane == 0) {
                pred[par][0][warp] = s0;
                pred[par][1][warp] = s1;
                pred[par][2][warp] = s2;
            }
            acc0.zero();
            acc1.zero();
            acc2.zero();
            pend_b = b;
        };
        auto write_pending = [&]() {  // after a barrier
            if (pend_b >= 0 && tid == 0) {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0;
                for (int w = 0; w < NTHR / 32; w++) {
                    s0 += pred[par][0][w];
                    s1 += pred[par][1][w];
                    s2 += pred[par][2][w];
                }
                A.partials[((size_t)0 * A.B + pend_b) * grid + blockIdx.x] = s0;
                A.partials[((size_t)1 * A.B + pend_b) * grid + blockIdx.x] = s1;
                if (FUSE)
                    A.partials[((size_t)2 * A.B + pend_b) * grid + blockIdx.x] = s2;
            }
            pend_b = -1;
        };

        // the compiled form of each stage's butterflies for this pass's shape
        const int d0 = due_form<G>(0, A.is_low, A.hmask, cb), d1 = due_form<G>(1, A.is_low, A.hmask, cb),
                  d2 = due_form<G>(2, A.is_low, A.hmask, cb);
        bool ok = true;
        for (unsigned k = 0; k < niter; k++) {
            unsigned b, t, mid;
            int c4;
            tile_coords(k, b, t, mid, c4);
            const int s = (int)(k % NS);
            unsigned char *buf = sm + (size_t)s * NV * TB;
            bool sync_now = (k == 0);  // launch constants (qr) and the table need a barrier
            if ((int)b != cur_b) {  // new parameter point: its phase table and mixer angle
                sync_now = true;
                if (cur_b >= 0 && reduce)
                    stash(cur_b);
                tslot ^= 1;
                X.tab = tab + tslot * MAXTAB;
                if constexpr (MG) {  // this point's own graph
                    if (est[0] >= 0 || est[1] >= 0) {
                        views(b, curv);
                        launch_consts(tslot);
                        X.qr = &qr[tslot][0][0];
                        X.qrf = &qrf[tslot][0][0];
                    }
                }
                if constexpr (IS) {
                    // this point's cost phases of the thread's and the stage's terms
                    // (each thread writes and reads only its own per-thread entries)
                    if (cost_phase && est[0] >= 0) {
                        const double ang = ising_angle(b);
                        double q, dk[G::RB], qq;
                        ising_terms(0, est[0], q, dk, qq);
                        ptp[tid] = unit_phase<R>(ang * q);
                        for (int kk = 0; kk < G::RB; kk++)
                            ptp[(1 + kk) * NTHR + tid] = unit_phase<R>(ang * dk[kk]);
                        if (tid < (1 << G::RB))
                            qps[tslot][tid] = unit_phase<R>(ang * qq);
                    }
                    X.qp = &qps[tslot][0];
                } else if (A.pre_phase || (A.post & (POST_PHASE_CONJ | POST_PHASE))) {
                    const C *src = reinterpret_cast<const C *>(A.tab) + ((size_t)b * A.p + A.tab_layer) * A.tab_len;
                    C *dst = tab + tslot * MAXTAB;
                    for (int i = tid; i < A.tab_len; i += NTHR)
                        dst[i] = src[i];
                }
                const double2 csd = A.cs[(size_t)b * A.p + A.layer];
                const double cbv = csd.x, sbv = A.sign_s * csd.y;
                const bool shifted = fabs(sbv) > fabs(cbv);  // rotate by beta - pi/2 (Ising: cot form)
                X.cot = IS && shifted;
                X.tq = shifted ? (R)((IS ? cbv : -cbv) / sbv) : (R)(sbv / cbv);
                const double f = shifted ? sbv : cbv;
                double fj = 1.0, fn = 1.0;
                for (int i = 0; i < A.n; i++) {
                    if (i < A.j0)
                        fj *= f;
                    fn *= f;
                }
                X.f = (R)f;
                X.fn = (R)fn;
                X.fn2 = (R)(fn * fn);
                X.scale0 = (R)fj;
                if constexpr (FUSE) {  // the second layer's rotation
                    const double2 cs2 = A.cs[(size_t)b * A.p + A.layer2];
                    const double c2 = cs2.x, s2 = A.sign_s * cs2.y;
                    const bool sh2 = fabs(s2) > fabs(c2);
                    X.cot2 = IS && sh2;
                    X.tq2 = sh2 ? (R)((IS ? c2 : -c2) / s2) : (R)(s2 / c2);
                    X.f2 = (R)(sh2 ? s2 : c2);
                }
                cur_b = (int)b;
            }
            X.sv0 = reinterpret_cast<C *>(buf);
            X.sv1 = reinterpret_cast<C *>(buf + TB);
            X.tc = &tcs[IS ? 0 : s][0][0];
            X.tv = &tvs[IS ? s : 0][0][0];
            X.tp = &tps[IS ? s : 0][0];
            X.fixed = ((uint64_t)mid << cb) | ((uint64_t)(t >> midbits) << (A.s + hb));

            // No barrier between tiles unless a point starts: a warp may begin
            // this tile while others still store the previous one. The first
            // barrier inside the tile decides a missed tile for all threads
            // alike (stage work on an unfilled buffer only reads garbage).
            const bool late = !mbar_wait_bounded(&full[s], (k / NS) & 1u);
            if (sync_now) {
                compute_sync<NTHR>();
                write_pending();
            }

            C a[NR], l[NR];
            X.first = true;
            X.run = X.scale0;
            bool bad;
            X.run2 = (R)1;
            if (!FUSE && P.is_low) {
                run_stage_due<R, NV, 0, OPS, false, IS>(d0, P, X, a, l, acc0, acc1, acc2);
                X.first = false;
                bad = compute_sync_or<NTHR>(late || *reinterpret_cast<volatile int *>(&s_flag));
                if (!bad) {
                    run_stage_due<R, NV, 1, OPS, false, IS>(d1, P, X, a, l, acc0, acc1, acc2);
                    if (!P.skip_last)
                        compute_sync<NTHR>();
                }
            } else {  // a high pass (every fused pass is one)
                run_stage_due<R, NV, 1, OPS, false, IS>(d1, P, X, a, l, acc0, acc1, acc2);
                X.first = false;
                bad = compute_sync_or<NTHR>(late || *reinterpret_cast<volatile int *>(&s_flag));
            }
            if (bad) {  // a tile never arrived, or the producer gave up
                if (tid == 0) {
                    atomicExch(A.err, 1);
                    s_flag = 1;
                }
                ok = false;
                break;
            }
            if (FUSE) {  // layer `layer` ends in stage 2, layer2 starts there and ends in stage 1
                run_stage_due<R, NV, 2, OPS, true, IS>(d2, P, X, a, l, acc0, acc1, acc2);
                compute_sync<NTHR>();
                mix_stage_due<R, NV, 1, IS>(d1, P, X, a, l, acc2);
            } else if (!P.skip_last) {  // a low pass over the qubits of stages 0 and 1 only ends here
                run_stage_due<R, NV, 2, OPS, false, IS>(d2, P, X, a, l, acc0, acc1, acc2);
            }
            // results (if any) are in the buffer: hand it to the producer
            fence_proxy_async_smem();
            mbar_arrive(&done[s]);
        }
        if (ok && reduce && cur_b >= 0) {
            stash(cur_b);
            compute_sync<NTHR>();
            write_pending();
        }
        };
        const int fw = flag_word(A.load, A.pre_phase, A.pre_lambda, A.write, A.post);
        using std::integral_constant;
        bool compiled = false;
        auto run_if = [&](auto flc) {
            if (!compiled && fw == decltype(flc)::value) {
                compute(flc);
                compiled = true;
            }
        };
        if constexpr (std::is_same<R, float>::value && MODE == 1 && NV == 1) {
            run_if(integral_constant<int, FW_FWD_FIRST>{});
            run_if(integral_constant<int, FW_FWD_LAST>{});
            run_if(integral_constant<int, FW_FWD_ENERGY>{});
        }
        if constexpr (std::is_same<R, float>::value && MODE == 3 && NV == 1)
            run_if(integral_constant<int, FW_FWD_FUSED>{});
        if constexpr (std::is_same<R, float>::value && MODE == 1 && NV == 2) {
            run_if(integral_constant<int, FW_ADJ_FIRST>{});
            run_if(integral_constant<int, FW_ADJ_LAST>{});
        }
        if constexpr (std::is_same<R, float>::value && MODE == 3 && NV == 2)
            run_if(integral_constant<int, FW_ADJ_BOUNDARY>{});
        if (!compiled)
            compute(integral_constant<int, -1>{});
    }
    __syncthreads();
    if (s_flag)
        return;
    if (reduce)
        pass_final_reduce(A, total);
}

// ------------------------------------------------- cluster low pass
// The adjoint's low pass over 14 qubits by a cluster of 4 CTAs (complex64,
// one parameter point). Cluster tile t is the 2^14 contiguous amplitudes
// t * 2^14 ...; CTA r of the cluster loads the slice whose qubits 12, 13
// equal r and applies the butterflies of qubits 0..11 in register stages 0,
// 1 and 2 as a plain low pass does. Stage 2 holds local bits 8..11 in
// registers; after its butterflies every thread stores each register into
// the shared memory of the CTA q whose slice has qubits 10, 11 = q (the
// register's local bits 10, 11), at local bits 10, 11 = r. Each CTA then
// holds the slice with qubits 10, 11 = its rank, qubits 12, 13 at local bits
// 10, 11, applies their butterflies in stage 3 (the stage-2 layout) and TMA-
// stores that slice. Two mbarriers per buffer order the exchange across the
// cluster: xl (every CTA has read its stage-2 registers, so its buffer may
// be overwritten) and xw (every CTA's stores into this buffer are done).
// Each CTA arrives once on every CTA's barrier (count 4) with release
// semantics at cluster scope and waits with acquire. All waits are bounded;
// a cluster barrier at the end keeps every CTA's shared memory alive while a
// peer may still reach it.
constexpr int CLUSTER_CTAS = 4;  // 2 qubits across the cluster

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_index()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// shared::cluster address of the same shared-memory location in CTA `cta`
__device__ __forceinline__ uint32_t map_to_cta(uint32_t addr, uint32_t cta)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(cta));
    return r;
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (clock64() - t0 > WAIT_BUDGET_CYCLES)
            return false;
    }
}
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void st_async_cluster4(uint32_t addr, float4 v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
                 : "memory");
}

// asynchronous store into a cluster CTA's shared memory that counts its
// bytes on that CTA's mbarrier (complete_tx) when they have landed
__device__ __forceinline__ void st_async_cluster(uint32_t addr, float2 v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "f"(v.x), "f"(v.y), "r"(bar)
                 : "memory");
}

// MODE 0: mixer only; 1: the first adjoint pass (phi loaded alone, lambda =
// O phi formed in stage 0). A.tiles counts 2^12-amplitude slices (2^(n-12)).
template <int MODE>
__global__ void __maxnreg__((Geo<float, 2>::MAXREG))
    k_cpass(const __grid_constant__ CUtensorMap ld0, const __grid_constant__ CUtensorMap ld1,
            const __grid_constant__ CUtensorMap st0, const __grid_constant__ CUtensorMap st1,
            const __grid_constant__ PassArgs A)
{
    using R = float;
    using G = Geo<float, 2>;
    using C = float2;
    constexpr bool OPS = MODE != 0;
    constexpr int NR = 1 << G::RB, NS = G::NSTAGE, NTHR = G::NTHR, RB = G::RB, NTB = G::T - G::RB;
    constexpr uint32_t TB = (uint32_t)tile_bytes<float, 2>();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ __align__(8) uint64_t full[NS], done[NS], xl[NS], xw[NS];
    __shared__ double pred[32];
    __shared__ int s_flag;
    __shared__ int obs_w[MAXK];
    __shared__ int tcs[NS][2][16];
    __shared__ int ptc[2 * (RB + 1) * NTHR];
    __shared__ int qr[2][32];
    __shared__ float qrf[2][32];

    const int tid = threadIdx.x;
    const uint32_t rank = cluster_ctarank();
    const unsigned cid = cluster_index(), ncl = cluster_count();
    uint64_t *obs_nbr = reinterpret_cast<uint64_t *>(sm + (size_t)NS * 2 * TB);
    const unsigned ctiles = (unsigned)A.tiles / CLUSTER_CTAS;
    const unsigned niter = cid < ctiles ? (ctiles - cid + ncl - 1) / ncl : 0;

    if (tid == 0) {
        s_flag = *reinterpret_cast<volatile int *>(A.err) ? 1 : 0;
        for (int q = 0; q < NS; q++) {
            mbar_init(&full[q], 1);
            mbar_init(&done[q], NTHR);
            mbar_init(&xl[q], CLUSTER_CTAS);
            mbar_init(&xw[q], 1);  // one local arrive with the expected bytes
        }
        fence_barrier_init();
    }
    if (OPS) {
        for (int i = tid; i < A.obs.K * MAXN; i += blockDim.x)
            obs_nbr[i] = A.obs.nbr[i / MAXN][i % MAXN];
        if (tid < MAXK)
            obs_w[tid] = A.obs.w[tid];
    }
    __syncthreads();
    cluster_barrier();  // every CTA's mbarriers are initialised before any remote arrive
    const bool skip = s_flag != 0;

    // O's launch constants for stage 0 (lambda = O phi); local bit L is qubit L
    if (OPS && !skip && tid < NTHR) {
        auto wgt = [&](int u, int v) -> int {
            int w = 0;
            for (int c = 0; c < A.obs.K; c++)
                w += obs_w[c] * (int)((obs_nbr[c * MAXN + u] >> v) & 1ull);
            return w;
        };
        int q = 0;
        for (int j = 0; j < NTB; j++)
            for (int j2 = 0; j2 < j; j2++)
                if (((tid >> j) & 1) && ((tid >> j2) & 1))
                    q -= 2 * wgt(G::thr(0, j), G::thr(0, j2));
        ptc[(RB + 1) * NTHR + tid] = q;
        for (int kk = 0; kk < RB; kk++) {
            int dk = 0;
            for (int j = 0; j < NTB; j++)
                if ((tid >> j) & 1)
                    dk -= 2 * wgt(G::reg(0, kk), G::thr(0, j));
            ptc[(RB + 1 + 1 + kk) * NTHR + tid] = dk;
        }
        if (tid < (1 << RB)) {
            int qq = 0;
            for (int kk = 0; kk < RB; kk++)
                for (int k2 = 0; k2 < kk; k2++)
                    if (((tid >> kk) & 1) && ((tid >> k2) & 1))
                        qq -= 2 * wgt(G::reg(0, kk), G::reg(0, k2));
            qr[1][tid] = qq;
            qrf[1][tid] = (float)qq;
        }
    }
    // fixed bits of this CTA's slice of cluster tile k
    auto slice_fixed = [&](unsigned k) -> uint64_t {  // within the point's state
        const uint64_t ct = (uint64_t)cid + (uint64_t)k * ncl;
        return (ct << 14) | ((uint64_t)rank << 12);
    };

    bool ok = !skip;
    if (!skip && tid >= NTHR) {
        // ------------------------------------------------------ producer
        const int lane = tid - NTHR;
        long long last_fill[NS];
        for (int q = 0; q < NS; q++)
            last_fill[q] = -1;
        auto fill = [&](unsigned k) {
            const int q = (int)(k % NS);
            if (OPS) {  // O(f) and h_L(f) of the slice (local bit L = qubit L)
                const uint64_t f = slice_fixed(k);
                int hs = 0, os = 0;
                for (int c = 0; c < A.obs.K; c++) {
                    const uint64_t *nb = obs_nbr + c * MAXN;
                    if (lane < G::T)
                        hs += obs_w[c] * (__popcll(nb[lane]) - 2 * __popcll(nb[lane] & f));
                    for (int u = lane; u < A.n; u += 32)
                        if ((f >> u) & 1ull)
                            os += obs_w[c] * __popcll(nb[u] & ~f);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    os += __shfl_xor_sync(0xffffffffu, os, o);
                if (lane < G::T)
                    tcs[q][1][lane] = hs;
                if (lane == 0)
                    tcs[q][1][15] = os;
            }
            __syncwarp();
            if (lane != 0)
                return;
            last_fill[q] = (long long)k;
            const int ct = A.tile0 + (int)(cid + k * ncl);
            unsigned char *buf = sm + (size_t)q * 2 * TB;
            mbar_arrive_expect_tx(&full[q], (uint32_t)A.nvec_io * TB);
            tma_load_5d(buf, &ld0, &full[q], 0, 0, 0, (int)rank, ct);
            if (A.nvec_io == 2)
                tma_load_5d(buf + TB, &ld1, &full[q], 0, 0, 0, (int)rank, ct);
        };
        for (unsigned k = 0; k < (unsigned)NS && k < niter; k++)
            fill(k);
        for (unsigned k = 0; k < niter && ok; k++) {
            const int q = (int)(k % NS);
            int good = 1;
            if (lane == 0) {
                good = mbar_wait_bounded(&done[q], (k / NS) & 1u) && !*reinterpret_cast<volatile int *>(&s_flag);
                if (good) {
                    const int ct = A.tile0 + (int)(cid + k * ncl);
                    unsigned char *buf = sm + (size_t)q * 2 * TB;
                    tma_store_5d(&st0, buf, 0, 0, (int)rank, 0, ct);
                    tma_store_5d(&st1, buf + TB, 0, 0, (int)rank, 0, ct);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    if (k + NS < niter)
                        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                }
            }
            good = __shfl_sync(0xffffffffu, good, 0);
            if (!good) {
                ok = false;
                break;
            }
            if (k + NS < niter)
                fill(k + NS);
        }
        if (lane == 0) {
            if (!ok) {
                atomicExch(A.err, 1);
                s_flag = 1;
                for (int q = 0; q < NS; q++)
                    if (last_fill[q] >= 0)
                        mbar_wait_bounded(&full[q], (unsigned)((last_fill[q] / NS) & 1));
            }
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        }
    } else if (!skip) {
        // ------------------------------------------------------- compute
        const PassRegs P{A.n, A.s, A.is_low, A.hmask, A.load, 0, A.pre_lambda, 1, 0, A.j0, 0, A.amp0};
        Acc<R> acc0, acc1, acc2;
        acc0.zero();
        acc1.zero();
        acc2.zero();
        StageCtx<R> X;
        X.ptc = ptc;
        X.qr = &qr[0][0];
        X.qrf = &qrf[0][0];
        X.s = A.s;
        X.cb = A.cb;
        X.tid = tid;
        X.amp0 = (R)A.amp0;
        X.cot = X.cot2 = false;
        {
            const double2 csd = A.cs[A.layer];
            const double cbv = csd.x, sbv = A.sign_s * csd.y;
            const bool shifted = fabs(sbv) > fabs(cbv);
            X.tq = shifted ? (R)(-cbv / sbv) : (R)(sbv / cbv);
            const double f = shifted ? sbv : cbv;
            double fj = 1.0, fn = 1.0;
            for (int i = 0; i < A.n; i++) {
                if (i < A.j0)
                    fj *= f;
                fn *= f;
            }
            X.f = (R)f;
            X.fn = (R)fn;
            X.fn2 = (R)(fn * fn);
            X.scale0 = (R)fj;
        }
        const uint32_t sb2 = G::swz(stage_base<G, 2>((uint32_t)tid));
        constexpr uint32_t LOW2 = split_low<G, 2>();
        const uint32_t sbh2 = sb2 & ~LOW2, sbl2 = sb2 & LOW2;
        // Software pipeline: stage 3 of tile k-1 (whose pushed quarters landed
        // while this CTA ran stages 0 and 1 of tile k) comes before stage 2 of
        // tile k, so the exchange's latency overlaps local work.
        R run_after2 = X.scale0;  // f^(j0 + 12): the same for every tile
        // the tile whose xl this CTA has signalled but whose incoming quarters
        // it has not yet waited for: peers may still be writing into it
        long long open_tile = -1;
        auto finish = [&](unsigned kp) -> bool {  // stage 3 of tile kp
            const int q = (int)(kp % NS);
            const bool got = mbar_wait_bounded(&xw[q], (kp / NS) & 1u);
            if (compute_sync_or<NTHR>(!got))
                return false;
            open_tile = -1;
            C a[NR], l[NR];
            C *sv0 = reinterpret_cast<C *>(sm + (size_t)q * 2 * TB);
            C *sv1 = reinterpret_cast<C *>(sm + (size_t)q * 2 * TB + TB);
            load_regs<R, 2, 2>(sv0, sb2, a);
            load_regs<R, 2, 2>(sv1, sb2, l);
            R run3 = run_after2;
            mix_regs<R, 2, 3>(P, X.cb, X.tq, X.f, run3, a, l, acc0);
            store_regs<R, 2, 2>(sv0, sb2, a);
            store_regs<R, 2, 2>(sv1, sb2, l);
            fence_proxy_async_smem();
            mbar_arrive(&done[q]);
            return true;
        };
        long long pending = -1;
        for (unsigned k = 0; k < niter; k++) {
            const int q = (int)(k % NS);
            const uint32_t par = (k / NS) & 1u;
            unsigned char *buf = sm + (size_t)q * 2 * TB;
            X.sv0 = reinterpret_cast<C *>(buf);
            X.sv1 = reinterpret_cast<C *>(buf + TB);
            X.tc = &tcs[q][0][0];
            const bool late = !mbar_wait_bounded(&full[q], par);
            if (k == 0)
                compute_sync<NTHR>();  // launch constants
            C a[NR], l[NR];
            X.first = true;
            X.run = X.scale0;
            run_stage<R, 2, 0, OPS>(P, X, a, l, acc0, acc1, acc2);
            X.first = false;
            if (compute_sync_or<NTHR>(late || *reinterpret_cast<volatile int *>(&s_flag))) {
                ok = false;
                break;
            }
            run_stage<R, 2, 1, OPS>(P, X, a, l, acc0, acc1, acc2);
            if (pending >= 0 && !finish((unsigned)pending)) {
                ok = false;
                break;
            }
            pending = -1;
            compute_sync<NTHR>();
            // stage 2: local bits 8..11, then the exchange
            load_regs<R, 2, 2>(X.sv0, sb2, a);
            load_regs<R, 2, 2>(X.sv1, sb2, l);
            fence_proxy_async_smem();  // these reads precede the peers' asynchronous stores
            compute_sync<NTHR>();      // this CTA's stage-2 reads are done
            if (tid < CLUSTER_CTAS)
                mbar_arrive_remote(map_to_cta(smem_u32(&xl[q]), (uint32_t)tid));
            open_tile = (long long)k;
            mix_regs<R, 2, 2>(P, X.cb, X.tq, X.f, X.run, a, l, acc0);
            run_after2 = X.run;
            const bool wl = mbar_wait_cluster_bounded(&xl[q], par);
            if (compute_sync_or<NTHR>(!wl)) {
                ok = false;
                break;
            }
            if (tid == 0)  // 4 quarters x 2 vectors land here, each with its byte count
                mbar_arrive_expect_tx(&xw[q], 2 * TB);
            // 16-byte stores: lane bit 0 is local bit 0, so a lane pair holds
            // two neighbouring amplitudes of every register; one shuffle per
            // register pair gives the even lane register m's pair and the odd
            // lane register m+1's (both go to the same CTA: bits 10, 11 agree)
            const uint32_t base0 = smem_u32(X.sv0), base1 = smem_u32(X.sv1), xwa = smem_u32(&xw[q]);
            const bool odd = tid & 1;
#pragma unroll
            for (int m = 0; m < NR; m += 2) {
                const uint32_t idx = smem_index<G, 2>(sbh2, sbl2, odd ? m + 1 : m) & ~1u;
                const uint32_t dst_cta = (idx >> 10) & 3u;
                const uint32_t dst = ((idx & ~(3u << 10)) | (rank << 10)) * (uint32_t)sizeof(C);
                const uint32_t bar = map_to_cta(xwa, dst_cta);
                const C sa = odd ? a[m] : a[m + 1], sl = odd ? l[m] : l[m + 1];
                C ra, rl;
                ra.x = __shfl_xor_sync(0xffffffffu, sa.x, 1);
                ra.y = __shfl_xor_sync(0xffffffffu, sa.y, 1);
                rl.x = __shfl_xor_sync(0xffffffffu, sl.x, 1);
                rl.y = __shfl_xor_sync(0xffffffffu, sl.y, 1);
                const float4 va = odd ? make_float4(ra.x, ra.y, a[m + 1].x, a[m + 1].y)
                                      : make_float4(a[m].x, a[m].y, ra.x, ra.y);
                const float4 vl = odd ? make_float4(rl.x, rl.y, l[m + 1].x, l[m + 1].y)
                                      : make_float4(l[m].x, l[m].y, rl.x, rl.y);
                st_async_cluster4(map_to_cta(base0 + dst, dst_cta), va, bar);
                st_async_cluster4(map_to_cta(base1 + dst, dst_cta), vl, bar);
            }
            pending = (long long)k;
        }
        if (ok && pending >= 0 && !finish((unsigned)pending))
            ok = false;
        if (!ok && tid == 0) {
            atomicExch(A.err, 1);
            s_flag = 1;
            // peers that passed this tile's xl may have asynchronous stores in
            // flight into this CTA: give them time to land before it leaves
            if (open_tile >= 0)
                mbar_wait_bounded(&xw[(int)(open_tile % NS)], (unsigned)((open_tile / NS) & 1));
        }
        // this CTA's dE/dbeta partial (slot 0)
        double s0 = acc0.get();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        if ((tid & 31) == 0)
            pred[tid >> 5] = s0;
        compute_sync<NTHR>();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NTHR / 32; w++)
                t += pred[w];
            A.partials[blockIdx.x] = t;
        }
    }
    __syncthreads();
    cluster_barrier();  // no CTA leaves while a peer may still address its shared memory
    if (s_flag || skip)
        return;
    pass_final_reduce(A, (unsigned)gridDim.x);
}

// ------------------------------------------------------ parameter tables
// The factor dropped by one tan/cot butterfly of the (inverse, sign = -1)
// mixer: cos beta if |sin| <= |cos| else sign * sin beta. Mirrors the choice
// the pass kernel makes from the same (cos, sin) pair.
__device__ __forceinline__ double butterfly_factor(double cn, double sn, double sign)
{
    const double s = sign * sn;
    return fabs(s) > fabs(cn) ? s : cn;
}

__device__ __forceinline__ double ipow(double f, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; i++)
        r *= f;
    return r;
}

// Three phase tables per (point, layer), each exp(-i ((gamma_l c) mod 2 pi))
// for c = 0..tab_len-1 computed in FP64 and rounded once:
//   tab[0]: exact, for the whole-circuit kernel;
//   tab[1]: times f_{l-1}^n, the factor the previous layer's n tan/cot
//           butterflies left on the state (forward passes);
//   tab[2]: conjugated and times f'_l^n for the inverse layer (adjoint).
// cs[b][l] = (cos beta_l, sin beta_l) in FP64.
template <typename R>
__global__ void k_params(int B, int p, int tab_len, int n, const double *__restrict__ gamma,
                         const double *__restrict__ beta, typename CT<R>::T *__restrict__ tab,
                         double2 *__restrict__ cs)
{
    using C = typename CT<R>::T;
    const double TWO_PI = 6.283185307179586476925286766559;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)B * p * tab_len;
    if (i < N) {
        const long long bl = i / tab_len;
        const int c = (int)(i - bl * tab_len);
        const int l = (int)(bl % p);
        double ang = fmod(gamma[bl] * (double)c, TWO_PI);
        if (ang < 0.0)
            ang += TWO_PI;
        double sn, cn;
        sincos(ang, &sn, &cn);
        double fs = 1.0;
        if (l > 0) {
            double bs, bc;
            sincos(beta[bl - 1], &bs, &bc);
            fs = ipow(butterfly_factor(bc, bs, 1.0), n);
        }
        double bs, bc;
        sincos(beta[bl], &bs, &bc);
        const double fb = ipow(butterfly_factor(bc, bs, -1.0), n);
        tab[i] = mkc<C>((R)cn, (R)(-sn));
        tab[N + i] = mkc<C>((R)(cn * fs), (R)(-sn * fs));
        tab[2 * N + i] = mkc<C>((R)(cn * fb), (R)(sn * fb));
    }
    if (i < (long long)B * p) {
        double sn, cn;
        sincos(beta[i], &sn, &cn);
        cs[i] = make_double2(cn, sn);
    }
}

// --------------------------------------------- whole circuit in one CTA
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

// O(x) of an Ising function, term by term in FP64
__device__ __forceinline__ double ising_direct(const IsingFn *F, int n, uint32_t x)
{
    double v = 0.0;
    for (int u = 0; u < n; u++) {
        const bool xu = (x >> u) & 1u;
        if (xu)
            v += F->h[u];
        for (int w = u + 1; w < n; w++)
            if ((bool)((x >> w) & 1u) != xu)
                v += F->W[u][w];
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
    // Ising plans: C(x) in FP64 for every basis state (after the table slot)
    const bool ising = A.icost != nullptr;
    double *cx = reinterpret_cast<double *>(tab + MAXTAB);
    auto cost_value = [&](int x) -> double { return ising ? cx[x] : (double)cut_direct(A.cost, n, (uint32_t)x); };
    auto obs_value = [&](int x) -> R {
        return ising ? (R)ising_direct(A.iobs, n, (uint32_t)x) : (R)cut_direct(A.obs, n, (uint32_t)x);
    };

    if (ising)
        for (int x = tid; x < N; x += NT)
            cx[x] = ising_direct(A.icost, n, (uint32_t)x);
    for (int x = tid; x < N; x += NT)
        phi[x] = mkc<C>((R)A.amp0, (R)0);
    for (int l = 0; l < A.p; l++) {
        __syncthreads();
        if (!ising) {
            const C *src = reinterpret_cast<const C *>(A.tab) + ((size_t)b * A.p + l) * A.tab_len;
            for (int i = tid; i < A.tab_len; i += NT)
                tab[i] = src[i];
        }
        const double2 cs = A.cs[(size_t)b * A.p + l];
        const R c = (R)cs.x, s = (R)cs.y;
        __syncthreads();
        if (ising) {  // exp(-i gamma_l C(x)), the angle in FP64
            const double gl = A.gam[(size_t)b * A.p + l];
            for (int x = tid; x < N; x += NT)
                phi[x] = cmul(phi[x], unit_phase<R>(-gl * cx[x]));
        } else {
            for (int x = tid; x < N; x += NT)
                phi[x] = cmul(phi[x], tab[cut_direct(A.cost, n, (uint32_t)x)]);
        }
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
        e += (double)((phi[x].x * phi[x].x + phi[x].y * phi[x].y) * obs_value(x));
    block_sum2<NT>(e, dummy, red);
    if (tid == 0)
        A.out[(size_t)b * A.out_stride] = e;
    if (A.mode != SMALL_GRAD)
        return;

    for (int x = tid; x < N; x += NT) {
        const R o = obs_value(x);
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
        if (l > 0 && !ising) {
            const C *src = reinterpret_cast<const C *>(A.tab) + ((size_t)b * A.p + l) * A.tab_len;
            for (int i = tid; i < A.tab_len; i += NT)
                tab[i] = src[i];
        }
        __syncthreads();
        const double gl = ising ? A.gam[(size_t)b * A.p + l] : 0.0;
        for (int x = tid; x < N; x += NT) {
            const double cv = cost_value(x);
            gg += (double)((R)cv * im_conj_mul(lam[x], phi[x]));
            if (l > 0) {
                const C t = ising ? unit_phase<R>(-gl * cv) : tab[(int)cv];
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

// ------------------------------------- uneven batch of small graphs
// One CTA per graph (n <= 13 for complex64, <= 12 for complex128), the whole
// p-layer circuit and the fused energy in shared memory. Each CTA reads its
// graph's masks from a device descriptor and builds its own phase factors
// exp(-i ((gamma_l c) mod 2 pi)) in FP64, so graphs of different n and |E|
// share one launch.
template <typename R>
__global__ void __launch_bounds__(256) k_small_multi(const SmallGraph *__restrict__ graphs, int G, int p, int obs,
                                                      const double *__restrict__ gamma,
                                                      const double *__restrict__ beta, double *__restrict__ energy)
{
    using C = typename CT<R>::T;
    constexpr int NT = 256;
    extern __shared__ __align__(16) unsigned char smem_multi[];
    __shared__ double red[2][32];
    __shared__ uint64_t s_cost[MAXN], s_obs[MAXK * MAXN];
    __shared__ int s_w[MAXK];
    const int g = blockIdx.x, tid = threadIdx.x;
    if (g >= G)
        return;
    const SmallGraph &D = graphs[g];
    const int n = D.n, N = 1 << n, half = N >> 1, K = D.K[obs], tab_len = D.tab_len;
    for (int i = tid; i < MAXN; i += NT)
        s_cost[i] = D.cost[i];
    for (int i = tid; i < K * MAXN; i += NT)
        s_obs[i] = D.obs[obs][i / MAXN][i % MAXN];
    if (tid < MAXK)
        s_w[tid] = D.w[obs][tid];
    C *phi = reinterpret_cast<C *>(smem_multi);
    C *tab = phi + N;
    const double TWO_PI = 6.283185307179586476925286766559;
    const double amp0 = rsqrt((double)N);
    for (int x = tid; x < N; x += NT)
        phi[x] = mkc<C>((R)amp0, (R)0);
    for (int l = 0; l < p; l++) {
        __syncthreads();
        const double gl = gamma[(size_t)D.gi * p + l];
        for (int c = tid; c < tab_len; c += NT) {
            double ang = fmod(gl * (double)c, TWO_PI);
            if (ang < 0.0)
                ang += TWO_PI;
            double sn, cn;
            sincos(ang, &sn, &cn);
            tab[c] = mkc<C>((R)cn, (R)(-sn));
        }
        double sb, cbv;
        sincos(beta[(size_t)D.gi * p + l], &sb, &cbv);
        const R c = (R)cbv, s = (R)sb;
        __syncthreads();
        for (int x = tid; x < N; x += NT) {
            int cv = 0;
            for (int u = 0; u < n; u++)
                cv += ((x >> u) & 1) ? __popcll(s_cost[u] & ~(uint64_t)x) : 0;
            phi[x] = cmul(phi[x], tab[cv]);
        }
        for (int q = 0; q < n; q++) {
            __syncthreads();
            for (int j = tid; j < half; j += NT) {
                const int x0 = ((j >> q) << (q + 1)) | (j & ((1 << q) - 1));
                bfly(phi[x0], phi[x0 | (1 << q)], c, s);
            }
        }
    }
    __syncthreads();
    double e = 0.0, dummy = 0.0;
    for (int x = tid; x < N; x += NT) {
        int v = 0;
        for (int k = 0; k < K; k++) {
            int cut = 0;
            for (int u = 0; u < n; u++)
                cut += ((x >> u) & 1) ? __popcll(s_obs[k * MAXN + u] & ~(uint64_t)x) : 0;
            v += s_w[k] * cut;
        }
        e += (double)((phi[x].x * phi[x].x + phi[x].y * phi[x].y) * (R)v);
    }
    block_sum2<NT>(e, dummy, red);
    if (tid == 0)
        energy[D.gi] = e;
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

// Low qubits 0..L-1 all transformed by register stages 0 and 1: a low pass
// over at most L qubits needs no third stage.
template <typename G>
constexpr int two_stage_low_bits()
{
    uint32_t m = 0;
    for (int st = 0; st < 2; st++)
        for (int k = 0; k < G::RB; k++)
            if ((G::own(st) >> k) & 1)
                m |= 1u << G::reg(st, k);
    int L = 0;
    while (L < G::T && ((m >> L) & 1))
        L++;
    return L;
}

int low_two_stage_bits(bool c128, int nv)
{
    if (c128)
        return nv == 2 ? two_stage_low_bits<Geo<double, 2>>() : two_stage_low_bits<Geo<double, 1>>();
    return nv == 2 ? two_stage_low_bits<Geo<float, 2>>() : two_stage_low_bits<Geo<float, 1>>();
}

void pass_geometry(bool c128, int nv, int *T, int *CB, int *HB)
{
    if (c128) {
        *T = nv == 2 ? Geo<double, 2>::T : Geo<double, 1>::T;
        *CB = nv == 2 ? Geo<double, 2>::CB : Geo<double, 1>::CB;
        *HB = nv == 2 ? Geo<double, 2>::HB : Geo<double, 1>::HB;
    } else {
        *T = nv == 2 ? Geo<float, 2>::T : Geo<float, 1>::T;
        *CB = nv == 2 ? Geo<float, 2>::CB : Geo<float, 1>::CB;
        *HB = nv == 2 ? Geo<float, 2>::HB : Geo<float, 1>::HB;
    }
}

int device_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) ==
                                                       cudaSuccess && v > 0)
            sms = v;
        else
            return 152;
    }
    return sms;
}

int pass_grid(long long total_tiles)
{
    const long long g = device_sms();
    return (int)(total_tiles < g ? total_tiles : g);
}

int launch_params(bool c128, int B, int p, int tab_len, int n, const double *d_gamma, const double *d_beta,
                  void *d_tab, double2 *d_cs, cudaStream_t st)
{
    const long long total = (long long)B * p * (tab_len > 1 ? tab_len : 1);
    const int grid = (int)((total + 255) / 256);
    if (c128)
        k_params<double><<<grid, 256, 0, st>>>(B, p, tab_len, n, d_gamma, d_beta, (double2 *)d_tab, d_cs);
    else
        k_params<float><<<grid, 256, 0, st>>>(B, p, tab_len, n, d_gamma, d_beta, (float2 *)d_tab, d_cs);
    return (int)cudaGetLastError();
}

template <typename R, int NV, int MODE>
static int launch_pass_ops(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                           cudaStream_t st)
{
    const size_t smem = pass_smem_total<R, NV, (MODE >= 4)>();
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e =
            cudaFuncSetAttribute(k_pass<R, NV, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return (int)e;
        attr_done = true;
    }
    k_pass<R, NV, MODE><<<grid, Geo<R, NV>::NTHR + 32, smem, st>>>(m0, m1, a);
    return (int)cudaGetLastError();
}

// passes without a pre- or post-operation run the lean instantiation; a batch
// of different graphs the per-point one; a fused pass (one graph, high qubits
// only) its own
template <typename R, int NV>
static int launch_pass_t(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid, cudaStream_t st)
{
    if (a.tiles < 1 || (a.tiles & (a.tiles - 1)))  // the kernel splits tile indices with shifts
        return (int)cudaErrorInvalidValue;
    const bool ops = a.pre_phase || a.pre_lambda || a.post || a.fuse;
    if (a.icost) {  // Ising plan: every pass (its layers may use the cot form)
        if (!a.iobs || !a.gam || a.pt)
            return (int)cudaErrorInvalidValue;
        if (a.fuse)
            return a.is_low ? (int)cudaErrorInvalidValue : launch_pass_ops<R, NV, 5>(m0, m1, a, grid, st);
        return ops ? launch_pass_ops<R, NV, 4>(m0, m1, a, grid, st) : launch_pass_ops<R, NV, 6>(m0, m1, a, grid, st);
    }
    if (!ops)
        return launch_pass_ops<R, NV, 0>(m0, m1, a, grid, st);
    if (a.fuse)
        return a.pt || a.is_low ? (int)cudaErrorInvalidValue : launch_pass_ops<R, NV, 3>(m0, m1, a, grid, st);
    return a.pt ? launch_pass_ops<R, NV, 2>(m0, m1, a, grid, st) : launch_pass_ops<R, NV, 1>(m0, m1, a, grid, st);
}

int launch_pass(bool c128, int nv_kernel, const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                cudaStream_t st)
{
    if (c128)
        return nv_kernel == 2 ? launch_pass_t<double, 2>(m0, m1, a, grid, st)
                              : launch_pass_t<double, 1>(m0, m1, a, grid, st);
    return nv_kernel == 2 ? launch_pass_t<float, 2>(m0, m1, a, grid, st)
                          : launch_pass_t<float, 1>(m0, m1, a, grid, st);
}

template <int MODE>
static int launch_cpass_t(const CUtensorMap *maps, const PassArgs &a, cudaStream_t st)
{
    const size_t smem = pass_smem_total<float, 2>();
    static bool attr_done = false;
    static int max_clusters[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64)
        return (int)(e != cudaSuccess ? e : cudaErrorInvalidDevice);
    if (!attr_done) {
        e = cudaFuncSetAttribute(k_cpass<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return (int)e;
        attr_done = true;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CLUSTER_CTAS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(Geo<float, 2>::NTHR + 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (!max_clusters[dev]) {  // clusters of 4 that fit at once (one CTA per SM)
        cfg.gridDim = dim3(CLUSTER_CTAS * 64);
        int c = 0;
        e = cudaOccupancyMaxActiveClusters(&c, k_cpass<MODE>, &cfg);
        if (e != cudaSuccess)
            return (int)e;
        if (c < 1)
            return (int)cudaErrorInvalidConfiguration;
        max_clusters[dev] = c;
    }
    const int ctiles = a.tiles / CLUSTER_CTAS;
    const int clusters = ctiles < max_clusters[dev] ? ctiles : max_clusters[dev];
    cfg.gridDim = dim3(CLUSTER_CTAS * clusters);
    e = cudaLaunchKernelEx(&cfg, k_cpass<MODE>, maps[0], maps[1], maps[2], maps[3], a);
    return (int)(e != cudaSuccess ? e : cudaGetLastError());
}

int launch_cluster_pass(const CUtensorMap *maps, const PassArgs &a, cudaStream_t st)
{
    if (a.B != 1 || a.tiles < CLUSTER_CTAS || (a.tiles & (a.tiles - 1)) || a.post || a.fuse || a.pt || a.icost ||
        !a.is_low)
        return (int)cudaErrorInvalidValue;
    return a.pre_lambda ? launch_cpass_t<1>(maps, a, st) : launch_cpass_t<0>(maps, a, st);
}

size_t small_smem_bytes(bool c128, int n, int mode, bool ising)
{
    const size_t amp = c128 ? 16 : 8;
    return ((mode == SMALL_GRAD ? 2 : 1) * ((size_t)1 << n) + MAXTAB) * amp + (ising ? ((size_t)1 << n) * 8 : 0);
}

int small_max_qubits(bool c128, int mode)
{
    // largest n whose state(s) plus the phase table fit the opt-in shared memory
    int n = 1;
    while (n < 20 && small_smem_bytes(c128, n + 1, mode, false) <= 200 * 1024)
        n++;
    return n;
}

int launch_small(bool c128, const SmallArgs &a, int B, cudaStream_t st)
{
    const size_t smem = small_smem_bytes(c128, a.n, a.mode, a.icost != nullptr);
    if (smem > 227 * 1024)
        return (int)cudaErrorInvalidValue;
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

// ------------------------------------------------ exported statevector
// The passes leave psi~(x) = i^|x| psi'(x) where psi' is the state of the
// circuit with every mixer layer l whose |sin beta_l| > |cos beta_l| rotated
// by beta_l - pi/2 instead of beta_l. With K such layers
//   psi = (-i)^(n K) (X^n)^K psi',
// so psi(x) = (-i)^(nK) i^(-|y|) psi~(y), y = x with all bits flipped when K
// is odd, else y = x. In place; for odd K each thread handles a pair (x, ~x).
// Ising plans never rotate by beta_l - pi/2 (noshift): K = 0.
template <typename R>
__global__ void k_untwist(typename CT<R>::T *psi, int n, const double2 *cs, int p, int noshift)
{
    using C = typename CT<R>::T;
    int K = 0;
    for (int l = 0; l < p && !noshift; l++)
        K += fabs(cs[l].y) > fabs(cs[l].x) ? 1 : 0;
    const int ph = (4 - ((n * K) & 3)) & 3;  // (-i)^(nK) = i^ph
    auto turn = [](C v, int e) -> C {          // v * i^e
        e &= 3;
        return e == 0 ? v : e == 1 ? mkc<C>(-v.y, v.x) : e == 2 ? mkc<C>(-v.x, -v.y) : mkc<C>(v.y, -v.x);
    };
    const uint64_t N = 1ull << n, full = N - 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (K & 1) {
        for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N / 2; x += stride) {
            const uint64_t y = x ^ full;
            const C vx = psi[x], vy = psi[y];
            psi[x] = turn(vy, ph - __popcll(y));
            psi[y] = turn(vx, ph - __popcll(x));
        }
    } else {
        for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += stride)
            psi[x] = turn(psi[x], ph - __popcll(x));
    }
}

// ------------------------------------------------------- maximum cut
// C_max = max_x C(x) by exhaustion with no memory traffic: each thread takes
// blocks of 32 states x0 | r (r over qubits 0..4) and evaluates them with the
// base-plus-deltas form of eval_cut. Only x with the top bit clear are
// visited (C(x) = C(~x), and the smallest maximiser has that bit clear). The
// result is packed as (value << 35) | (2^35 - 1 - x), so one atomicMax keeps
// the largest value and, among equal values, the smallest x, in any order.
__global__ void __launch_bounds__(256) k_maxcut(const __grid_constant__ CostFn cost, int n,
                                                unsigned long long *key)
{
    const int nb = n - 1;
    auto pack = [](int v, uint64_t x) { return ((unsigned long long)v << 35) | ((1ull << 35) - 1ull - x); };
    unsigned long long best = 0;
    if (nb < 5) {
        if (blockIdx.x == 0 && threadIdx.x < (1u << nb)) {
            const uint64_t x = threadIdx.x;
            int c = 0;
            for (int cl = 0; cl < cost.K; cl++) {
                int s = 0;
                for (int u = 0; u < n; u++)
                    s += ((x >> u) & 1ull) ? __popcll(cost.nbr[cl][u] & ~x) : 0;
                c += cost.w[cl] * s;
            }
            best = pack(c, x);
        }
    } else {
        const uint64_t blocks = 1ull << (nb - 5);
        const int gp[5] = {0, 1, 2, 3, 4};
        for (uint64_t blk = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; blk < blocks;
             blk += (uint64_t)gridDim.x * blockDim.x) {
            const uint64_t x0 = blk << 5;
            int v[32];
            eval_cut<5>(cost, n, x0, gp, v);
#pragma unroll
            for (int m = 0; m < 32; m++) {
                const unsigned long long q = pack(v[m], x0 | (uint64_t)m);
                best = q > best ? q : best;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, best, o);
        best = q > best ? q : best;
    }
    if ((threadIdx.x & 31) == 0 && best)
        atomicMax(key, best);
}

int launch_maxcut(const CostFn &cost, int n, unsigned long long *d_key, cudaStream_t st)
{
    k_maxcut<<<4 * device_sms(), 256, 0, st>>>(cost, n, d_key);
    return (int)cudaGetLastError();
}

// ----------------------------------------------------------- sampling
// Inverse-CDF sampling from |psi(x)|^2 (the twisted frame has the same
// moduli). Chunk c holds amplitudes [c 2^SB, (c+1) 2^SB). sums[c] is the FP64
// chunk total (fixed-order block reduction); an exclusive scan turns it into
// the cumulative mass before the chunk; then one warp per sample finds the
// chunk by binary search and the amplitude inside it by a lane scan. Sample k
// is the smallest x whose cumulative mass exceeds u_k * total (the last index
// if rounding leaves none).
constexpr int SAMPLE_BITS = 12;

template <typename R>
__global__ void __launch_bounds__(256) k_sample_chunks(const typename CT<R>::T *psi, int n, double *sums)
{
    __shared__ double red[2][32];
    const int cb = n < SAMPLE_BITS ? n : SAMPLE_BITS;
    const uint64_t nchunks = 1ull << (n - cb), len = 1ull << cb;
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        double s = 0.0;
        for (uint64_t i = threadIdx.x; i < len; i += blockDim.x) {
            const typename CT<R>::T a = psi[c * len + i];
            s += (double)a.x * (double)a.x + (double)a.y * (double)a.y;
        }
        double z = 0.0;
        block_sum2<256>(s, z, red);
        if (threadIdx.x == 0)
            sums[c] = s;
        __syncthreads();
    }
}

// exclusive scan of `count` doubles in place, one block of 1024 threads,
// each thread a contiguous segment; writes the grand total to *total
__global__ void __launch_bounds__(1024) k_sample_scan(double *v, uint64_t count, double *total)
{
    __shared__ double seg[1024];
    const uint64_t per = (count + 1023) / 1024;
    const uint64_t lo = threadIdx.x * per, hi = lo + per < count ? lo + per : count;
    double s = 0.0;
    for (uint64_t i = lo; i < hi; i++)
        s += v[i];
    seg[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int t = 0; t < 1024; t++) {
            const double c = seg[t];
            seg[t] = run;
            run += c;
        }
        *total = run;
    }
    __syncthreads();
    double run = seg[threadIdx.x];
    for (uint64_t i = lo; i < hi; i++) {
        const double c = v[i];
        v[i] = run;
        run += c;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_sample_draw(const typename CT<R>::T *psi, int n, const double *prefix,
                                                     const double *total, int K, const double *u,
                                                     unsigned long long *x_out, int *cut_out,
                                                     const __grid_constant__ CostFn cost)
{
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int cb = n < SAMPLE_BITS ? n : SAMPLE_BITS;
    const uint64_t nchunks = 1ull << (n - cb), len = 1ull << cb, N = 1ull << n;
    const uint64_t per = len >= 32 ? len / 32 : 1;  // amplitudes per lane
    for (int k = warp; k < K; k += nwarps) {
        const double t = u[k] * *total;
        uint64_t lo = 0, hi = nchunks;  // last chunk with prefix <= t
        while (hi - lo > 1) {
            const uint64_t mid = lo + (hi - lo) / 2;
            if (prefix[mid] <= t)
                lo = mid;
            else
                hi = mid;
        }
        const uint64_t c = lo;
        const double rem = t - prefix[c];
        // lane sums, then an inclusive warp scan in lane order
        const uint64_t base = c * len + (uint64_t)lane * per;
        double s = 0.0;
        if ((uint64_t)lane * per < len)
            for (uint64_t i = 0; i < per; i++) {
                const typename CT<R>::T a = psi[base + i];
                s += (double)a.x * (double)a.x + (double)a.y * (double)a.y;
            }
        double inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o)
                inc += y;
        }
        const unsigned over = __ballot_sync(0xffffffffu, inc > rem && (uint64_t)lane * per < len);
        uint64_t x;
        if (over) {
            const int L = __ffs(over) - 1;
            const double before = __shfl_sync(0xffffffffu, inc - s, L);
            x = c * len + (uint64_t)L * per + per - 1;  // fallback: the lane's last amplitude
            if (lane == L) {
                double run = before;
                for (uint64_t i = 0; i < per; i++) {
                    const typename CT<R>::T a = psi[base + i];
                    run += (double)a.x * (double)a.x + (double)a.y * (double)a.y;
                    if (run > rem) {
                        x = base + i;
                        break;
                    }
                }
            }
            x = __shfl_sync(0xffffffffu, x, L);
        } else {
            x = c + 1 < nchunks ? (c + 1) * len - 1 : N - 1;  // rounding left the target past the chunk
        }
        if (lane == 0) {
            x_out[k] = x;
            if (cut_out) {
                int v = 0;
                for (int cl = 0; cl < cost.K; cl++) {
                    int s = 0;
                    for (int q = 0; q < n; q++)
                        s += ((x >> q) & 1ull) ? __popcll(cost.nbr[cl][q] & ~x) : 0;
                    v += cost.w[cl] * s;
                }
                cut_out[k] = v;
            }
        }
    }
}

size_t sample_chunk_count(int n) { return (size_t)1 << (n < SAMPLE_BITS ? 0 : n - SAMPLE_BITS); }

int launch_sample(bool c128, const void *psi, int n, double *d_sums, double *d_total, int K, const double *d_u,
                  unsigned long long *d_x, int *d_cut, const CostFn &cost, cudaStream_t st)
{
    const uint64_t nchunks = sample_chunk_count(n);
    const int g1 = (int)(nchunks < (uint64_t)(8 * device_sms()) ? nchunks : (uint64_t)(8 * device_sms()));
    const int g3 = (K + 7) / 8 < 4 * device_sms() ? (K + 7) / 8 : 4 * device_sms();
    if (c128)
        k_sample_chunks<double><<<g1, 256, 0, st>>>((const double2 *)psi, n, d_sums);
    else
        k_sample_chunks<float><<<g1, 256, 0, st>>>((const float2 *)psi, n, d_sums);
    k_sample_scan<<<1, 1024, 0, st>>>(d_sums, nchunks, d_total);
    if (c128)
        k_sample_draw<double><<<g3, 256, 0, st>>>((const double2 *)psi, n, d_sums, d_total, K, d_u, d_x, d_cut, cost);
    else
        k_sample_draw<float><<<g3, 256, 0, st>>>((const float2 *)psi, n, d_sums, d_total, K, d_u, d_x, d_cut, cost);
    return (int)cudaGetLastError();
}

int launch_untwist(bool c128, void *psi, int n, const double2 *cs, int p, int noshift, cudaStream_t st)
{
    const int grid = 4 * device_sms();
    if (c128)
        k_untwist<double><<<grid, 256, 0, st>>>((double2 *)psi, n, cs, p, noshift);
    else
        k_untwist<float><<<grid, 256, 0, st>>>((float2 *)psi, n, cs, p, noshift);
    return (int)cudaGetLastError();
}

size_t small_multi_smem_bytes(bool c128, int max_n, int max_tab)
{
    return (((size_t)1 << max_n) + (size_t)max_tab) * (c128 ? 16 : 8);
}

int launch_small_multi(bool c128, const SmallGraph *d_graphs, int G, int p, int obs, int max_n, int max_tab,
                       const double *d_gamma, const double *d_beta, double *d_energy, cudaStream_t st)
{
    const size_t smem = small_multi_smem_bytes(c128, max_n, max_tab);
    cudaError_t e;
    if (c128) {
        e = cudaFuncSetAttribute(k_small_multi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return (int)e;
        k_small_multi<double><<<G, 256, smem, st>>>(d_graphs, G, p, obs, d_gamma, d_beta, d_energy);
    } else {
        e = cudaFuncSetAttribute(k_small_multi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return (int)e;
        k_small_multi<float><<<G, 256, smem, st>>>(d_graphs, G, p, obs, d_gamma, d_beta, d_energy);
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

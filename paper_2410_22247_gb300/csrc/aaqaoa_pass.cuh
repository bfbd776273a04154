// sm_103a pass kernel of the AA-QAOA hot path (k_pass) and the device
// helpers the other kernels share; included by aaqaoa_kernels.cu and by the
// units that instantiate the passes (aaqaoa_pass_*.cu).
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
//    layer's first pass (or, with layer-boundary fusion, into the end of the
//    pass that ends layer l-1); the reduction (energy), lambda = O psi,
//    dE/dgamma and the inverse cost phase are folded into the last stage of a
//    pass. C(x) is computed exactly in integers: per thread one cut value by
//    popcount over neighbour masks, then each of the thread's 2^RB amplitudes
//    by flipping register bits (cut change of a flipped vertex, corrected for
//    flipped neighbour pairs). The phase is a table lookup T_l[C(x)] of
//    exp(-i gamma_l c) built in FP64 with the argument reduced mod 2 pi.
//  * Reductions accumulate per thread in FP64 and are summed in a fixed order
//    by the last block of the grid, so results are bit-reproducible.
//
// Every wait on an mbarrier is bounded by a clock64 budget; on expiry the
// block sets the device error flag, waits once more (bounded) for its own TMA
// copies and returns without touching global memory.
#pragma once

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

// The turnaround pass (POST_LAMBDA) leaves phi as loaded and stores lambda
// scaled to match it (complex64; complex128 passes are FP64-bound and store
// both vectors, the extra state would cost them spills).
template <typename R>
constexpr bool turn_keeps_phi = std::is_same<R, float>::value;

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
    // turnaround pass (POST_LAMBDA, turn_keeps_phi): phi is not stored back,
    // the stored lambda carries kap = f^(2 j0 - n) instead (see run_stage),
    // and the pass's dE/dbeta sums are multiplied by 1/kap once per point
    R kap;
    double ikap;
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
    // the register-bit pair terms of function e in this pass's cut stage are
    // all zero (the usual case: few couplings among one stage's bits), so
    // their per-amplitude additions (and the Ising phases' factors) are skipped
    bool qz[2] = {false, false};
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
__device__ __forceinline__ void cut_int(const int *tc, const int *pt, const int *qr, bool qz, int tid,
                                        int (&v)[1 << G::RB])
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
    if (!qz)
#pragma unroll
        for (int m = 1; m < (1 << RB); m++)
            v[m] += qr[m];
}

// cut values as multipliers of type R (exact: integers below 2^24)
template <typename G, typename R, int ST>
__device__ __forceinline__ void cut_real(const int *tc, const int *pt, const int *qr, const float *qrf, bool qz,
                                         int tid, R (&v)[1 << G::RB])
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
        if (!qz)
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
        if (!qz)
#pragma unroll
            for (int m = 1; m < (1 << RB); m++)
                iv[m] += qr[m];
#pragma unroll
        for (int m = 0; m < (1 << RB); m++)
            v[m] = (R)iv[m];
    }
}

// Ising plans: the same quadratic decomposition with real couplings and
// fields. Values O(x) of the thread's 2^RB states from constants rounded
// once to R (tile: tc[15] = O(f), tc[L] = h_L(f); thread: pt; stage: q).
template <typename G, typename R, int ST>
__device__ __forceinline__ void ising_vals(const R *tc, const R *pt, const R *q, bool qz, int tid,
                                           R (&v)[1 << G::RB])
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
    if (!qz)
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
__device__ __forceinline__ void ising_phases(const C *tp, const C *pp, const C *qp, bool qz, int tid,
                                             C (&P)[1 << G::RB])
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
    // (complex128 keeps the loop unconditional: the branch there costs the
    // 255-register forward pass spills)
    if (!(qz && std::is_same<C, float2>::value))
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

template <typename R, int NV, int ST, bool COT, int DUE, bool PHI = false>
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
            if constexpr (NV == 2 && !PHI) {
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
        if constexpr (NV == 2 && !PHI) {
            const R q = ((ipp[0].x + ipp[0].y) + (ipp[1].x + ipp[1].y)) - ((ipn[0].x + ipn[0].y) + (ipn[1].x + ipn[1].y));
            gb = fma(q, sc * sc, gb);
        }
        sc *= f;
    }
    run = sc;
    if constexpr (NV == 2 && !PHI)
        acc.add(gb);
}

// cot (Ising plans only, decided per layer) selects the butterfly form once
// for the whole stage, outside the unrolled loops
template <typename R, int NV, int ST, bool IS = false, int DUE = -1, bool PHI = false>
__device__ __forceinline__ void mix_regs(const PassRegs &A, int cb, R tq, R f, R &run,
                                         typename CT<R>::T (&a)[1 << Geo<R, NV>::RB],
                                         typename CT<R>::T (&l)[1 << Geo<R, NV>::RB], Acc<R> &acc,
                                         bool cot = false)
{
    if (IS && cot)
        mix_regs_form<R, NV, ST, true, DUE, PHI>(A, cb, tq, f, run, a, l, acc);
    else
        mix_regs_form<R, NV, ST, false, DUE, PHI>(A, cb, tq, f, run, a, l, acc);
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

    // the stage a pass starts with: stage 0 of a low pass, or stage 1 of a
    // complex64 high pass (the generating pass of a forward sweep may be one)
    constexpr bool MAY_START = ST == 0 || (ST == 1 && std::is_same<R, float>::value);
    if (MAY_START && X.first && !A.load) {  // |+>^n in the twisted frame: 2^(-n/2) i^|x|
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
        if constexpr (NV == 2)  // lambda exists unless this pass forms it
            if (!(OPS && X.first && A.pre_lambda) && !(OPS && (A.post & POST_LAMBDA)))
                load_regs<R, NV, ST>(X.sv1, sb, l);
    }

    // cut-function constants: function 0 is C (cost), 1 the observable O
    const int *tc0 = X.tc, *tc1 = X.tc + 16;
    const int *pt0 = X.ptc + X.tid, *pt1 = X.ptc + (RB + 1) * G::NTHR + X.tid;
    // the values O_e(x) of the thread's states (real; exact integers for cut functions)
    auto values = [&](int e, R (&v)[NR]) {
        if constexpr (IS)
            ising_vals<G, R, ST>(X.tv + 16 * e, X.ptv + e * (RB + 1) * G::NTHR + X.tid, X.qv + 32 * e, X.qz[e], X.tid,
                                 v);
        else
            cut_real<G, R, ST>(e ? tc1 : tc0, e ? pt1 : pt0, X.qr + 32 * e, X.qrf + 32 * e, X.qz[e], X.tid, v);
    };
    // the cost layer's phase factors of the thread's states (this pass's table)
    auto phases = [&](C (&P)[NR]) {
        if constexpr (IS) {
            ising_phases<G, C, ST>(X.tp, X.ptp + X.tid, X.qp, X.qz[0], X.tid, P);
        } else {
            int cv[NR];
            cut_int<G, ST>(tc0, pt0, X.qr, X.qz[0], X.tid, cv);
#pragma unroll
            for (int m = 0; m < NR; m++)
                P[m] = X.tab[cv[m]];
        }
    };

    if (OPS && MAY_START && X.first && A.pre_phase) {
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

    if (NV == 2 && OPS && (A.post & POST_LAMBDA))  // phi alone (lambda is formed below)
        mix_regs<R, NV, ST, IS, DUE, true>(A, X.cb, X.tq, X.f, X.run, a, l, acc0, X.cot);
    else
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
        if constexpr (NV == 2) {
            if (A.post & POST_LAMBDA) {  // lambda = O phi of the exact final state
                // Mixing this pass's q qubits forward (t), rescaling by f^n and
                // mixing them back (-t) multiplies phi by f^n (1 + t^2)^q =
                // f^(n - 2q) = 1/kap: the phi this pass would store is the one
                // it loaded times 1/kap. It is not stored; lambda is stored
                // times kap, so every later product of the two is unchanged
                // (complex64; complex128 stores both as they are).
#pragma unroll
                for (int m = 0; m < NR; m++) {
                    const R w = turn_keeps_phi<R> ? ov[m] * X.kap : ov[m];
                    l[m] = mkc<C>(a[m].x * w, a[m].y * w);
                }
            }
        }
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
            if (LAST || !(OPS && (A.post & POST_LAMBDA)))  // lambda exists from the last stage on
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
    if (!(turn_keeps_phi<R> && NV == 2 && (A.post & POST_LAMBDA)))  // the turnaround keeps the loaded phi
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
__device__ inline void pass_final_reduce(const PassArgs &A, unsigned total)
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
constexpr int FW_TURN = flag_word(1, 0, 0, 1, POST_REDUCE | POST_RESCALE | POST_LAMBDA);  // forward ends, adjoint starts

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
    // C for the phase of a layer's first forward pass (its first stage: 0 for
    // a low pass, 1 for the generating high pass), for the next layer's
    // phase in a fused forward pass and for the gradient and inverse phase of
    // the last adjoint pass of a layer (last stage); O for
    // lambda = O phi (first stage of the first adjoint pass) and for the
    // energy (last stage of the last forward pass).
    int est[2] = {-1, -1};
    if (OPS) {
        if (A.pre_phase)  // in the pass's first stage
            est[0] = A.is_low ? 0 : 1;
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
                    d += F->W[v][u];  // symmetric: lanes read one row
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
        // g_u(f) adds one precomputed chunk sum per 6 bits of f (IsingFn::G:
        // a walk over the set bits of f waited on each load in turn).
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
                    double g = 0.0;  // g_u(f): one chunk sum per 6 bits of f
                    const double d = isd[e][u];
#pragma unroll
                    for (int c = 0; c < ISING_CHUNKS; c++)
                        if (6 * c < A.n)
                            g += F->G[c][(f >> (6 * c)) & 63u][u];
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
                    if (!(turn_keeps_phi<R> && NV == 2 && (A.post & POST_LAMBDA)))  // the turnaround keeps phi
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
                if (turn_keeps_phi<R> && NV == 2 && (P.post & POST_LAMBDA))  // lambda carried kap
                    s2 *= X.ikap;
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
                    if constexpr (turn_keeps_phi<R> && NV == 2) {
                        X.kap = (R)(fj * fj / fn);  // f^(2 j0 - n), j0 = n - q
                        X.ikap = fn / (fj * fj);
                    }
                    if constexpr (FUSE) {  // the second layer's rotation
                        const double2 cs2 = A.cs[(size_t)b * A.p + A.layer2];
                        const double c2 = cs2.x, s2 = (A.sign2 != 0.0 ? A.sign2 : A.sign_s) * cs2.y;
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
                    if constexpr (OPS) {  // this point's register-bit pair terms, now visible
#pragma unroll
                        for (int e = 0; e < 2; e++) {
                            bool z = true;
                            for (int m = 1; m < NR; m++)
                                z = z && (IS ? X.qv[32 * e + m] == (R)0 : X.qr[32 * e + m] == 0);
                            X.qz[e] = z;
                        }
                    }
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
        // cut-function modes 1 and 3 and their Ising counterparts 4 and 5
        constexpr bool F32 = std::is_same<R, float>::value;
        if constexpr (F32 && (MODE == 1 || MODE == 4) && NV == 1) {
            run_if(integral_constant<int, FW_FWD_FIRST>{});
            run_if(integral_constant<int, FW_FWD_LAST>{});
            run_if(integral_constant<int, FW_FWD_ENERGY>{});
        }
        if constexpr (F32 && (MODE == 3 || MODE == 5) && NV == 1)
            run_if(integral_constant<int, FW_FWD_FUSED>{});
        if constexpr (F32 && (MODE == 1 || MODE == 4) && NV == 2) {
            run_if(integral_constant<int, FW_ADJ_FIRST>{});
            run_if(integral_constant<int, FW_ADJ_LAST>{});
        }
        if constexpr (F32 && (MODE == 3 || MODE == 5) && NV == 2) {
            run_if(integral_constant<int, FW_ADJ_BOUNDARY>{});
            run_if(integral_constant<int, FW_TURN>{});
        }
        if (!compiled)
            compute(integral_constant<int, -1>{});
    }
    __syncthreads();
    if (s_flag)
        return;
    if (reduce)
        pass_final_reduce(A, total);
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

// Cut-function (MaxCut) plans: passes without a pre- or post-operation run
// the lean instantiation; a batch of different graphs the per-point one; a
// fused pass (one graph, high qubits only) its own.
template <typename R, int NV>
static int launch_pass_cut_t(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                             cudaStream_t st)
{
    if (a.tiles < 1 || (a.tiles & (a.tiles - 1)) || a.icost)  // the kernel splits tile indices with shifts
        return (int)cudaErrorInvalidValue;
    const bool ops = a.pre_phase || a.pre_lambda || a.post || a.fuse;
    if (!ops)
        return launch_pass_ops<R, NV, 0>(m0, m1, a, grid, st);
    if (a.fuse)
        return a.pt || a.is_low ? (int)cudaErrorInvalidValue : launch_pass_ops<R, NV, 3>(m0, m1, a, grid, st);
    return a.pt ? launch_pass_ops<R, NV, 2>(m0, m1, a, grid, st) : launch_pass_ops<R, NV, 1>(m0, m1, a, grid, st);
}

// Ising plans: every pass (its layers may use the cot form).
template <typename R, int NV>
static int launch_pass_ising_t(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                               cudaStream_t st)
{
    if (a.tiles < 1 || (a.tiles & (a.tiles - 1)) || !a.icost || !a.iobs || !a.gam || a.pt)
        return (int)cudaErrorInvalidValue;
    const bool ops = a.pre_phase || a.pre_lambda || a.post || a.fuse;
    if (a.fuse)
        return a.is_low ? (int)cudaErrorInvalidValue : launch_pass_ops<R, NV, 5>(m0, m1, a, grid, st);
    return ops ? launch_pass_ops<R, NV, 4>(m0, m1, a, grid, st) : launch_pass_ops<R, NV, 6>(m0, m1, a, grid, st);
}

}  // namespace aaq

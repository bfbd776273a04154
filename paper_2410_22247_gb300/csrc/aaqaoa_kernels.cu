// sm_103a kernels of the AA-QAOA hot path other than the tiled pass: the
// adjoint's cluster low pass, the whole-circuit kernels for small n and
// uneven batches, aggregation, export, parameter tables, maximum cut and
// sampling, with their launchers. The pass kernel and the shared device
// helpers are in aaqaoa_pass.cuh.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "aaqaoa_internal.h"
#include "aaqaoa_pass.cuh"

namespace aaq {

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

// the pass instantiations live in units of their own (aaqaoa_pass_*.cu), so
// that they compile in parallel
int launch_pass(bool c128, int nv_kernel, const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                cudaStream_t st)
{
    if (c128)
        return launch_pass_c128(nv_kernel, m0, m1, a, grid, st);
    if (a.icost)
        return nv_kernel == 2 ? launch_pass_c64_ising_adj(m0, m1, a, grid, st)
                              : launch_pass_c64_ising_fwd(m0, m1, a, grid, st);
    return nv_kernel == 2 ? launch_pass_c64_adj(m0, m1, a, grid, st) : launch_pass_c64_fwd(m0, m1, a, grid, st);
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

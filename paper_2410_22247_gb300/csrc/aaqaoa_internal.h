// Internal declarations shared by the host side (aaqaoa_host.cu) and the
// kernels (aaqaoa_pass.cuh, aaqaoa_pass_*.cu, aaqaoa_kernels.cu). Not part
// of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace aaq {

constexpr int MAXN = 34;   // qubits
constexpr int MAXK = 10;   // weight classes of a weighted cut function
constexpr int MAXTAB = 562; // |E| + 1 for K_34

// A weighted cut function O(x) = sum_c w[c] * sum_{edges (u,v) of class c} [x_u != x_v],
// stored as per-class vertex neighbour masks. H_C is the single class of all
// edges at weight 1; H_red groups the orbit representatives by weight.
struct CutFn {
    int K;
    int w[MAXK];
    uint64_t nbr[MAXK][MAXN];
};

// The cost function C(x) of the ansatz: one class at weight 1 for MaxCut;
// integer edge weights grouped into classes for weighted MaxCut.
using CostFn = CutFn;

// An Ising-form function O(x) = sum_{u<v} W[u][v] [x_u != x_v] + sum_u h[u] x_u
// with real couplings (W symmetric, zero where there is no edge) and real
// fields: the cost of an Ising plan, and its observables (H_red keeps one
// representative edge per edge orbit and one vertex per vertex orbit, each at
// orbit size times its weight or field).
constexpr int ISING_CHUNKS = (MAXN + 5) / 6;  // 6-bit chunks of a basis index
struct IsingFn {
    double W[MAXN][MAXN];  // symmetric
    double h[MAXN];
    // G[c][m][u] = sum of W[6c + j][u] over the set bits j of m: g_u(f) =
    // sum_{v in f} W_vu is one entry per 6-bit chunk of f, loads that do
    // not wait on each other, with a warp's vertices u on one row
    double G[ISING_CHUNKS][64][MAXN];
};

// Cut functions of one graph of a batch of graphs with the same n: the cost
// C(x) and the two observables (0 = H_C, 1 = H_red).
struct GraphFns {
    CutFn cost;
    CutFn obs[2];
};

// Operations of one tiled pass over the statevector(s).
enum PostOp : int {
    POST_REDUCE = 1,      // acc0 += |phi|^2 O(x)                 (energy)
    POST_RESCALE = 2,     // multiply by f^n: the stored final state is exact
    POST_GAMMA = 4,       // acc1 += C(x) Im(conj(lambda) phi)     (dE/dgamma)
    POST_PHASE_CONJ = 8,  // phi, lambda *= inverse-layer table    (undo cost layer)
    POST_PHASE = 16,      // phi *= forward table of layer tab_layer (next cost layer)
    POST_LAMBDA = 32,     // two-vector pass: lambda = O(x) phi formed after the energy
                          // (the pass's first mixer acts on phi alone: lambda does not
                          // exist before; the turnaround of a gradient evaluation;
                          // complex64: phi stays as loaded, lambda is stored scaled
                          // to match it)
};

struct PassArgs {
    int n;            // qubits
    int s;            // global bit of local high bit 0
    int cb;           // contiguous bits of a tile row (local bits 0..cb-1 = qubits 0..cb-1)
    int wide_rows;    // tensor map form: 1 when a row spans more than 128 bytes
    int is_low;       // tile is contiguous and its low bits are transformed here
    int hmask;        // which local high bits (bit j = local bit cb + j) get a butterfly
    int tiles;        // tiles per statevector = 2^(n - tile bits)
    int B;            // statevectors (parameter points) in this launch
    int chunk;        // 0: CTAs interleave tiles; else each CTA takes `chunk` consecutive tiles
    int skip_last;    // low pass whose qubits all lie in register stages 0 and 1 (no third stage)
    int load;         // 1: TMA-load the tile(s); 0: generate |+>^n
    int pre_phase;    // multiply by the cost-layer phase before any butterfly
    int pre_lambda;   // adjoint: load phi only and form lambda = O(x) phi first
    int write;        // TMA-store the tile(s) after the last stage
    int post;         // PostOp flags
    int nvec_io;      // vectors loaded (1 or 2)
    int layer;        // layer l (0-based): selects the phase table and (cos, sin)
    int tab_layer;    // layer whose phase table the pass applies (the next one when fused)
    int fuse;         // 1: after the last stage's operations, apply layer `layer2`'s mixer
                      //    to the same qubits (a layer boundary inside one pass)
    int layer2;       // the second layer of a fused pass
    int j0;           // butterflies of this layer applied by earlier passes (adjoint)
    int p;            // number of layers
    int tab_len;      // |E| + 1
    double sign_s;    // +1: exp(-i beta H_M); -1: its inverse
    double sign2;     // the second layer of a fused pass: the same, or 0 for sign_s
    double amp0;      // 2^(-n/2) for the generated |+>^n
    const void *tab;  // this pass's phase tables [B][p][tab_len]: forward-scaled or inverse
    const double2 *cs;  // [B][p] (cos beta_l, sin beta_l)
    double *partials; // [3][B][grid]
    unsigned *counter;  // last-block counter (zero between launches)
    double *out;      // [B][out_stride]
    int out_stride;
    int slot_idx[3];  // output index (within a point's row) of slot 0 / 1 / 2, or -1
    double slot_scale[3];  // slot 0: acc0 (energy or dE/dbeta_layer), 1: dE/dgamma, 2: dE/dbeta_layer2
    int *err;         // device error flag
    int drop_first_load;  // test hook: CTA 0 never loads its first tile (bounded wait expires)
    CutFn obs;        // observable of the reduction / lambda
    CostFn cost;      // C(x) for the phase and dE/dgamma
    const GraphFns *pt;  // non-null: point b is its own graph, pt[b] (obs and cost above unused)
    int pt_obs;          // which observable of pt[b]
    // Ising plans (real couplings and fields): the cost and the observable as
    // dense couplings, gamma per (point, layer); obs and cost above unused.
    // Their layers never drop a factor -iX: a layer with |sin| > |cos| uses
    // the cot form of the rotation instead.
    const IsingFn *icost;
    const IsingFn *iobs;
    const double *gam;   // [B][p]
    int tile0;           // cluster low pass: first cluster tile (point b of a batch starts at b * 2^(n-14))
};

// Whole-circuit kernel for states that fit one CTA's shared memory.
enum SmallMode : int { SMALL_ENERGY = 0, SMALL_GRAD = 1 };

struct SmallArgs {
    int n, p, tab_len, mode;
    int write_state;   // also store psi_p to `state`
    double amp0;
    const void *tab;
    const double2 *cs;
    double *out;       // [B][out_stride]
    int out_stride;
    void *state;       // [B][2^n] (optional)
    CutFn obs;
    CostFn cost;
    const IsingFn *icost;  // non-null: an Ising plan (obs and cost above unused)
    const IsingFn *iobs;
    const double *gam;     // [B][p]
};

// Device descriptor of one small graph in an uneven batch (whole circuit in
// one CTA): cost masks, and the masks and weights of both observables
// (index 0 = H_C, 1 = H_red).
struct SmallGraph {
    int gi;  // index of the graph in the batch: its (gamma, beta) row and energy slot
    int n, tab_len;
    int K[2];
    int w[2][MAXK];
    uint64_t cost[MAXN];
    uint64_t obs[2][MAXK][MAXN];
};

// Aggregation over a stored statevector.
struct AggArgs {
    int n;
    uint64_t chunks;     // number of 1024-amplitude chunks (per state)
    const void *state;
    double *partials;    // [T][grid]
    unsigned *counter;
    double *out_terms;   // per-term <Z_u Z_v>, or nullptr
    double *out_energy;  // accumulates sum_t w_t (1 - zz_t)/2 or sum |psi|^2 O(x)
    int num_terms;       // terms of this launch
    int term_u[64], term_v[64];
    double term_w[64];
    CutFn obs;           // fused mode
};

// Launchers (aaqaoa_kernels.cu, aaqaoa_pass_*.cu). They return a cudaError_t as int.
int tile_bits(bool c128);
void pass_geometry(bool c128, int nv, int *T, int *CB, int *HB);
int low_two_stage_bits(bool c128, int nv);
int device_sms();
int pass_grid(long long total_tiles);
int launch_params(bool c128, int B, int p, int tab_len, int n, const double *d_gamma, const double *d_beta,
                  void *d_tab, double2 *d_cs, cudaStream_t st);
int launch_pass(bool c128, int nv_kernel, const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a,
                int grid, cudaStream_t st);
// the pass instantiations, one unit each: complex64 cut-function plans
// forward and adjoint, complex64 Ising plans forward and adjoint,
// complex128 (both kinds)
int launch_pass_c64_fwd(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid, cudaStream_t st);
int launch_pass_c64_adj(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid, cudaStream_t st);
int launch_pass_c64_ising_fwd(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                              cudaStream_t st);
int launch_pass_c64_ising_adj(const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                              cudaStream_t st);
int launch_pass_c128(int nv_kernel, const CUtensorMap &m0, const CUtensorMap &m1, const PassArgs &a, int grid,
                     cudaStream_t st);
// The adjoint's complex64 low pass over 14 qubits by clusters of 4 CTAs: maps
// = {load phi, load lambda, store phi, store lambda}; one parameter point.
int launch_cluster_pass(const CUtensorMap *maps, const PassArgs &a, cudaStream_t st);
constexpr int CLUSTER_LOW_QUBITS = 14;
int launch_small(bool c128, const SmallArgs &a, int B, cudaStream_t st);
size_t small_smem_bytes(bool c128, int n, int mode, bool ising);
int small_max_qubits(bool c128, int mode);
int launch_agg_fused(bool c128, const AggArgs &a, cudaStream_t st, int grid);
int launch_agg_terms(bool c128, const AggArgs &a, cudaStream_t st, int grid);
int agg_grid(bool c128);
size_t small_multi_smem_bytes(bool c128, int max_n, int max_tab);
int launch_untwist(bool c128, void *psi, int n, const double2 *cs, int p, int noshift, cudaStream_t st);
int launch_maxcut(const CostFn &cost, int n, unsigned long long *d_key, cudaStream_t st);
size_t sample_chunk_count(int n);
int launch_sample(bool c128, const void *psi, int n, double *d_sums, double *d_total, int K, const double *d_u,
                  unsigned long long *d_x, int *d_cut, const CostFn &cost, cudaStream_t st);
int launch_small_multi(bool c128, const SmallGraph *d_graphs, int G, int p, int obs, int max_n, int max_tab,
                       const double *d_gamma, const double *d_beta, double *d_energy, cudaStream_t st);

}  // namespace aaq

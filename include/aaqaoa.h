/*
 * aaqaoa.h -- C ABI of the GB300 (sm_103a) AA-QAOA hot path.
 *
 * What it computes (Automorphism-Assisted QAOA, arXiv:2410.22247):
 *   |psi_p(gamma, beta)> = prod_{l=1..p} exp(-i beta_l H_M) exp(-i gamma_l H_C) |+>^n
 * (Eq. (1); layer 1 acts first on |+>^n, as Eq. (A2) writes the product out),
 * with the unweighted MaxCut cost H_C = 1/2 sum_{(i,j) in E} (1 - Z_i Z_j)
 * (Eq. for H_P with w_ij in {0, 1}; integer edge weights through
 * aaqaoa_prepare_weighted) and the mixer H_M = sum_i X_i, followed by
 * the cost expectation (F_p, Eq. (2)) aggregated over all 2^n amplitudes
 * with one of two observables:
 *   AAQAOA_OBS_FULL  H_C itself;
 *   AAQAOA_OBS_RED   H_red = 1/2 sum_m |S~_m| (1 - Z_{i_m} Z_{j_m}), one
 *                    representative edge per edge orbit weighted by the orbit
 *                    size (Sec. 5, equation for H_red). The ansatz is always
 *                    built from the full H_C; only the measured observable is
 *                    reduced, and <H_red> = <H_C> exactly (Eq. (exact)).
 *
 * Conventions: qubit i is bit i of the basis-state index (little-endian).
 * Amplitudes are complex64 (AAQAOA_C64: float re/im pairs) or complex128
 * (AAQAOA_C128: double re/im pairs); every reduction (energy, gradient,
 * <Z Z>) accumulates in FP64 and every phase gamma*C(x) is reduced mod 2*pi
 * in FP64 before it is rounded to the storage precision. The returned energy
 * is E = <psi| O |psi> (the expected cut, >= 0); minimising or maximising it is
 * the caller's business.
 *
 * Threading and streams: a plan is not thread-safe; calls on one plan must be
 * serialised by the caller. All device work of a plan is issued on the plan's
 * CUDA stream (set at prepare time or with aaqaoa_set_stream). Calls that
 * take host pointers synchronise that stream before they return; calls that
 * take device pointers only enqueue work.
 *
 * Errors: every int-returning entry point returns AAQAOA_OK (0) or a negative
 * AAQAOA_ERR_* code and never aborts the process. aaqaoa_strerror() gives a
 * fixed description of a code; aaqaoa_last_error_detail() gives the message
 * recorded by the last failing call on the calling thread.
 */
#ifndef AAQAOA_H
#define AAQAOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aaqaoa_plan aaqaoa_plan; /* opaque, owned by the library */

/* prepare() flags: amplitude precision */
#define AAQAOA_C64  0u
#define AAQAOA_C128 1u

/* observables */
#define AAQAOA_OBS_FULL 0
#define AAQAOA_OBS_RED  1

/* aggregation modes of aaqaoa_expect():
 *   FUSED      one FP64 sum of |psi_x|^2 O(x) folded into the last pass of the
 *              circuit (no extra read of the state);
 *   PERTERM    the estimator aggregation of Eq. (agg): one full pass over the
 *              amplitudes per ZZ term (|E| passes for H_C, |O_E| for H_red),
 *              the cost model whose term count the paper reduces;
 *   SINGLEPASS one pass over the stored state that evaluates all terms of
 *              the observable per amplitude (sum_x |psi_x|^2 O(x) with
 *              O(x) = sum_terms w [x_u != x_v]), i.e. the whole aggregation
 *              in a single read;
 *   PERORBIT   the same single read, named for H_red: every orbit
 *              representative's term (weighted by its orbit size) is
 *              accumulated per amplitude in one pass; per-edge or per-orbit
 *              <Z_u Z_v> values themselves come from aaqaoa_edge_zz. */
#define AAQAOA_AGG_FUSED      0
#define AAQAOA_AGG_PERTERM    1
#define AAQAOA_AGG_SINGLEPASS 2
#define AAQAOA_AGG_PERORBIT   AAQAOA_AGG_SINGLEPASS

/* error codes */
#define AAQAOA_OK               0
#define AAQAOA_ERR_INVALID_ARG  (-1) /* bad n, p, edge list, pointer or size      */
#define AAQAOA_ERR_BAD_ORBITS   (-2) /* orbit data do not partition the edges     */
#define AAQAOA_ERR_WORKSPACE    (-3) /* no workspace, or one too small/misaligned */
#define AAQAOA_ERR_CUDA         (-4) /* a CUDA call failed (detail recorded)      */
#define AAQAOA_ERR_TIMEOUT      (-5) /* a bounded device wait expired             */
#define AAQAOA_ERR_UNSUPPORTED  (-6) /* valid request the library does not serve */

#define AAQAOA_MAX_QUBITS 34

/*
 * aaqaoa_prepare -- validate a graph and its edge orbits, build a plan.
 *
 * n            number of vertices = qubits, 1 <= n <= 34.
 * num_edges    |E| >= 0.
 * edges        host, 2*num_edges int32: edge e joins edges[2e] and edges[2e+1].
 *              Vertices in [0, n); no self-loops; no repeated edge (in either
 *              orientation). Any order; the plan keeps the caller's edge
 *              indexing for orbit_rep / edge_orbit.
 * num_orbits   |O_E| (0 if no reduced observable is wanted).
 * orbit_rep    host, num_orbits int32: index (into edges) of the representative
 *              (i_m, j_m) of each orbit S~_m (Sec. 5). May be NULL if
 *              num_orbits == 0.
 * orbit_weight host, num_orbits int32: |S~_m| >= 1; must sum to num_edges.
 * edge_orbit   host, num_edges int32 or NULL: the orbit of each edge. When
 *              given, it must be a partition consistent with orbit_rep (each
 *              representative lies in its own orbit) and orbit_weight (class
 *              sizes). The library cannot check that the classes are true
 *              Aut(G) orbits (Algorithm 1); exactness of H_red relies on it.
 * p            number of QAOA layers, 1 <= p <= 64.
 * flags        AAQAOA_C64 or AAQAOA_C128.
 * stream       cudaStream_t (as void*) for all device work; NULL = legacy
 *              default stream.
 * out          receives the plan; *out is NULL on error.
 *
 * All host arrays are copied; the caller may free them on return. No device
 * memory is allocated: device buffers come from aaqaoa_set_workspace().
 * Errors: INVALID_ARG, BAD_ORBITS.
 */
int aaqaoa_prepare(int n, int num_edges, const int32_t *edges,
                   int num_orbits, const int32_t *orbit_rep, const int32_t *orbit_weight,
                   const int32_t *edge_orbit, int p, unsigned flags, void *stream,
                   aaqaoa_plan **out);

/*
 * aaqaoa_prepare_weighted -- aaqaoa_prepare for weighted MaxCut with integer
 * edge weights w_e >= 1: H_C = 1/2 sum_e w_e (1 - Z_u Z_v), so the phase uses
 * the weighted cut C(x) = sum_e w_e [x_u != x_v] and H_red keeps one
 * representative per class at weight |S~_m| * w_rep (Sec. 5 with the edge
 * weights carried along; orbits must come from weight-preserving
 * automorphisms). edge_weight: num_edges int32, or NULL for all 1 (then this
 * is aaqaoa_prepare). The total weight must not exceed 561 (the phase table
 * holds one entry per cut value): AAQAOA_ERR_UNSUPPORTED otherwise.
 * AAQAOA_ERR_BAD_ORBITS if edge_orbit puts edges of different weight in one
 * class. Plans with weights are not accepted by aaqaoa_prepare_multi.
 */
int aaqaoa_prepare_weighted(int n, int num_edges, const int32_t *edges, const int32_t *edge_weight, int num_orbits,
                            const int32_t *orbit_rep, const int32_t *orbit_weight, const int32_t *edge_orbit, int p,
                            unsigned flags, void *stream, aaqaoa_plan **out);

/*
 * aaqaoa_prepare_ising -- a plan for an Ising-form objective with real
 * couplings and fields, the generalisation the paper's conclusion names
 * (weighted MaxCut and more general Ising objectives with non-trivial
 * automorphism groups):
 *   H_C = sum_e w_e 1/2 (1 - Z_u Z_v) + sum_i h_i 1/2 (1 - Z_i),
 * whose diagonal is C(x) = sum_e w_e [x_u != x_v] + sum_i h_i x_i. The ansatz
 * is Eq. (1) with this H_C in the cost layer; E = <H_C> (or <H_red>).
 * edge_weight: num_edges doubles (any finite sign). field: n doubles, or NULL
 * for no fields. Edges, p, flags and the edge orbits are as for
 * aaqaoa_prepare; H_red keeps one representative edge per edge orbit at
 * |orbit| * w_rep and, with fields, one representative vertex per vertex
 * orbit at |orbit| * h_rep (vorbit_rep, vorbit_weight: num_vorbits int32
 * each; vertex_orbit: n int32 or NULL). Both kinds of orbits must come from
 * automorphisms that preserve the couplings and the fields (Eq. A3 then makes
 * <H_red> = <H_C>); edge_orbit / vertex_orbit, when given, are checked for
 * equal weights / fields within a class. Vertex orbits are required when
 * there are fields and edge orbits.
 * The cost phase exp(-i gamma C(x)) is built per amplitude from products of
 * unit phase factors whose angles are reduced in FP64; C(x) and the
 * observables are real (not exact integers). Ising plans support the fused
 * aggregation only: aaqaoa_expect with PERTERM/SINGLEPASS,
 * aaqaoa_aggregate_only, aaqaoa_max_cut, aaqaoa_sample and
 * aaqaoa_expect_static return AAQAOA_ERR_UNSUPPORTED. Every other call on a
 * plan (energies, gradients, batches, statevector, edge_zz, verify_orbits,
 * pass plans) works as for MaxCut.
 * Errors: INVALID_ARG (also a weight or field that is not finite),
 * BAD_ORBITS. Host arrays are copied; no device memory is allocated.
 */
int aaqaoa_prepare_ising(int n, int num_edges, const int32_t *edges, const double *edge_weight, const double *field,
                         int num_orbits, const int32_t *orbit_rep, const int32_t *orbit_weight,
                         const int32_t *edge_orbit, int num_vorbits, const int32_t *vorbit_rep,
                         const int32_t *vorbit_weight, const int32_t *vertex_orbit, int p, unsigned flags, void *stream,
                         aaqaoa_plan **out);

/*
 * aaqaoa_workspace_bytes -- device bytes needed for a workspace able to hold
 * `batch` statevectors (batch >= 1), with room for the adjoint gradient's
 * second statevector when with_grad != 0. Writes *bytes.
 */
int aaqaoa_workspace_bytes(const aaqaoa_plan *plan, int batch, int with_grad, size_t *bytes);

/*
 * aaqaoa_set_workspace -- hand the plan a device buffer (caller-owned; e.g. a
 * torch tensor) of at least aaqaoa_workspace_bytes(plan, batch, with_grad)
 * bytes, 256-byte aligned. The plan keeps the pointer until the next call or
 * aaqaoa_destroy; the caller must keep the memory alive meanwhile.
 * Errors: INVALID_ARG, WORKSPACE (too small / misaligned), CUDA.
 */
int aaqaoa_set_workspace(aaqaoa_plan *plan, void *device_ptr, size_t bytes, int batch, int with_grad);

/* aaqaoa_set_stream -- change the plan's CUDA stream (cudaStream_t as void*). */
int aaqaoa_set_stream(aaqaoa_plan *plan, void *stream);

/*
 * aaqaoa_expect -- E = <psi_p(gamma, beta)| O |psi_p(gamma, beta)>.
 *
 * gamma, beta  host, p doubles each.
 * observable   AAQAOA_OBS_FULL or AAQAOA_OBS_RED (RED needs num_orbits > 0).
 * agg_mode     AAQAOA_AGG_FUSED / PERTERM / SINGLEPASS (see above).
 * energy       host, 1 double.
 * Synchronises the plan's stream. Errors: INVALID_ARG, WORKSPACE, CUDA, TIMEOUT.
 */
int aaqaoa_expect(aaqaoa_plan *plan, const double *gamma, const double *beta,
                  int observable, int agg_mode, double *energy);

/*
 * aaqaoa_grad -- energy and its gradient by the adjoint method.
 *
 * With phi = psi_p and lambda = O psi_p, for l = p..1 the library applies the
 * inverse mixer and cost layers to both vectors and accumulates
 * dE/dbeta_l = 2 Im <lambda| H_M |phi> and dE/dgamma_l = 2 Im <lambda| H_C |phi>
 * (derivative of F_p, Eq. (2)). Two statevectors; the workspace must have
 * been set with with_grad != 0.
 * gamma, beta, dgamma, dbeta: host, p doubles each; energy: host, 1 double.
 * Synchronises the plan's stream.
 */
int aaqaoa_grad(aaqaoa_plan *plan, const double *gamma, const double *beta, int observable,
                double *energy, double *dgamma, double *dbeta);

/*
 * aaqaoa_expect_batch -- energies of B parameter points on the plan's graph.
 * gamma, beta: host, B*p doubles (point-major: point b uses gamma[b*p .. b*p+p-1]).
 * energy: host, B doubles. Points are processed in groups of the workspace's
 * batch capacity. Fused aggregation. Synchronises the plan's stream.
 */
int aaqaoa_expect_batch(aaqaoa_plan *plan, int B, const double *gamma, const double *beta,
                        int observable, double *energy);

/*
 * aaqaoa_grad_batch -- energy and adjoint gradient of B parameter points on
 * the plan's graph (multi-start optimisation, gradient landscapes), the
 * points of one wave sharing every launch. gamma, beta: host, B*p doubles
 * (point-major); energy: host, B doubles; dgamma, dbeta: host, B*p doubles
 * (point-major). Points are processed in waves of the workspace's batch
 * capacity, which must have been set with with_grad != 0 (two statevectors
 * per point). Synchronises the plan's stream.
 * Errors: INVALID_ARG (NULL pointer, B < 1), WORKSPACE, CUDA, TIMEOUT.
 */
int aaqaoa_grad_batch(aaqaoa_plan *plan, int B, const double *gamma, const double *beta, int observable,
                      double *energy, double *dgamma, double *dbeta);

/*
 * Device-pointer forms: the same computations with every argument already in
 * device memory. They only enqueue work on the plan's stream and return; the
 * results are valid once that stream has reached them. A device-side timeout
 * is reported by the next call of aaqaoa_sync().
 *
 * aaqaoa_expect_device: d_gamma, d_beta: B*p doubles; d_energy: B doubles
 *   (B <= the workspace's batch capacity). Fused aggregation.
 * aaqaoa_grad_device: d_gamma, d_beta: p doubles; d_out: 1 + 2p doubles laid
 *   out as [E, dE/dgamma_1..p, dE/dbeta_1..p].
 */
int aaqaoa_expect_device(aaqaoa_plan *plan, int B, const double *d_gamma, const double *d_beta,
                         int observable, double *d_energy);
int aaqaoa_grad_device(aaqaoa_plan *plan, const double *d_gamma, const double *d_beta,
                       int observable, double *d_out);
/* aaqaoa_grad_batch_device: d_gamma, d_beta: B*p doubles (point-major); d_out:
 *   B rows of 1 + 2p doubles, [E, dE/dgamma_1..p, dE/dbeta_1..p] per point
 *   (B <= the workspace's batch capacity; gradient workspace). */
int aaqaoa_grad_batch_device(aaqaoa_plan *plan, int B, const double *d_gamma, const double *d_beta,
                             int observable, double *d_out);

/* aaqaoa_sync -- wait for the plan's stream and report any device-side error. */
int aaqaoa_sync(aaqaoa_plan *plan);

/*
 * aaqaoa_edge_zz -- <Z_u Z_v> for every edge of the graph in one pass over the
 * final state (the per-term values that Eq. (agg) sums; equal within an edge
 * orbit by Eq. (A3)). zz: host, num_edges doubles, in the caller's edge order.
 */
int aaqaoa_edge_zz(aaqaoa_plan *plan, const double *gamma, const double *beta, double *zz);

/*
 * aaqaoa_verify_orbits -- debug check of the orbit data behind H_red. The
 * library cannot prove that the classes given to aaqaoa_prepare are orbits of
 * Aut(G) (Sec. 4, Algorithm 1); by Eq. (A3) every member of a true orbit has
 * the same <Z_u Z_v> as its representative at any angles. This call evaluates
 * all edge terms at (gamma, beta) (host arrays of p doubles, preferably
 * generic values) and compares each edge with the representative of its
 * class. Equality is necessary, not sufficient: a class that passes at one
 * angle set may still fail at another.
 * tol: largest accepted |<ZZ>_e - <ZZ>_rep| (>= 0; about 1e-5 for C64,
 *   1e-10 for C128). bad_orbit (host, 1 int): -1 on success, else the first
 *   class that fails.
 * Returns AAQAOA_ERR_BAD_ORBITS for a failing class, AAQAOA_ERR_INVALID_ARG
 * if the plan was prepared without edge_orbit (membership unknown).
 */
int aaqaoa_verify_orbits(aaqaoa_plan *plan, const double *gamma, const double *beta, double tol, int *bad_orbit);

/*
 * aaqaoa_max_cut -- C_max = max over all 2^n basis states of the cut count
 * C(x), the denominator of the approximation ratio F_p / C_max (Sec. 2), by
 * exhaustion on the device: no statevector is read (the workspace is only
 * needed for an 8-byte result). c_max (host, 1 int32); argmax (host, 1
 * uint64): the smallest x that attains it (bit i = vertex i on side 1).
 * Synchronises the plan's stream.
 */
int aaqaoa_max_cut(aaqaoa_plan *plan, int32_t *c_max, uint64_t *argmax);

/*
 * aaqaoa_sample -- K bitstrings drawn from the final-state distribution
 * |psi_p(x)|^2 (the measurement the paper's pipeline ends with, Sec. 5.4).
 * The uniform numbers are the caller's: u (host, K doubles in [0, 1)); sample
 * k is the smallest x whose cumulative probability sum_{y <= x} |psi_y|^2,
 * taken in index order and in FP64, exceeds u_k times the total. x_out (host,
 * K uint64); cut_out (host, K int32, or NULL): C(x) of each sample.
 * 1 <= K <= AAQAOA_SAMPLE_MAX per call. The state is left in the workspace
 * (aaqaoa_aggregate_only may follow). Errors: INVALID_ARG for K or u out of
 * range.
 */
#define AAQAOA_SAMPLE_MAX 65536
int aaqaoa_sample(aaqaoa_plan *plan, const double *gamma, const double *beta, int K, const double *u,
                  uint64_t *x_out, int32_t *cut_out);

/*
 * aaqaoa_statevector -- the final state psi_p itself, copied to host memory:
 * 2^n complex amplitudes in the plan's precision (interleaved re, im as float
 * for C64 or double for C128). host_out must hold 2^n * 8 (C64) or
 * 2^n * 16 (C128) bytes.
 */
int aaqaoa_statevector(aaqaoa_plan *plan, const double *gamma, const double *beta, void *host_out);

/*
 * aaqaoa_aggregate_only -- time-isolated aggregation: evaluate
 * <psi|O|psi> on the state left in the workspace by the last
 * aaqaoa_statevector / aaqaoa_edge_zz / non-fused aaqaoa_expect call, with
 * the given observable and aggregation mode, without re-running the circuit.
 * energy: host, 1 double. Synchronises the plan's stream.
 */
int aaqaoa_aggregate_only(aaqaoa_plan *plan, int observable, int agg_mode, double *energy);

/*
 * aaqaoa_expect_static -- aaqaoa_expect (fused aggregation) without a
 * workspace and without any device allocation by the library.
 *
 * The paper has no counterpart: this serves callers that cannot allocate
 * device memory at the point where they evaluate an energy -- for example code
 * that runs under a host application which owns every device allocation, or a
 * process that has used up its device-memory budget and still needs energies
 * of small graphs -- so they cannot provide a workspace.
 *
 * Device scratch (control words, phase tables, parameters, partial sums and
 * one statevector) lives in a file-scope static device array of 33 MiB
 * compiled into the library; every GPU that loads the library holds it until
 * the process exits. It fits one statevector of up to 2^22 complex64 or 2^21
 * complex128 amplitudes: n <= 22 for AAQAOA_C64, n <= 21 for AAQAOA_C128;
 * larger n returns AAQAOA_ERR_UNSUPPORTED with a message.
 *
 * The first call on a device looks up the array's device address (and so
 * makes the CUDA runtime load the library's device module); make that first
 * call before any stream capture. The address is kept for the life of the
 * process: it does not survive cudaDeviceReset (or anything else that
 * replaces the device's primary context), after which this entry point must
 * not be called again in that process. Every call shares the one array: the entry
 * point clears what must start at zero, but calls that overlap on the GPU
 * (other streams, other host threads, concurrent graph replays) race on it.
 *
 * plan: prepared graph (no workspace needed). gamma, beta: host, p doubles.
 * observable: AAQAOA_OBS_FULL or AAQAOA_OBS_RED. energy: host, 1 double.
 * Synchronises the plan's stream. Calls no cudaMalloc/cudaFree.
 */
int aaqaoa_expect_static(aaqaoa_plan *plan, const double *gamma, const double *beta, int observable,
                         double *energy);

/*
 * Uneven batches of graphs (many small instances of different n, one call).
 *
 * aaqaoa_graph_desc describes one graph exactly as the arguments of
 * aaqaoa_prepare (edges, optional orbit representatives and weights, and the
 * optional class of every edge, edge_orbit, NULL when not given).
 * aaqaoa_prepare_multi validates every graph (same rules and errors as
 * aaqaoa_prepare, the detail names the graph) and copies all host arrays.
 * Graphs that fit one CTA (n <= 13 for C64, n <= 12 for C128) are evaluated
 * together by one kernel launch; each larger graph runs the tiled passes.
 * The first aaqaoa_expect_multi call for an observable times a few ways of
 * spreading the large graphs over parallel CUDA streams (autotune; cached per
 * device and batch shape for the process; AAQAOA_AUTOTUNE=0 in the
 * environment skips the timing) and captures the whole evaluation into a
 * CUDA graph, which later calls replay.
 *
 * aaqaoa_multi_workspace_bytes / aaqaoa_multi_set_workspace: one caller-owned
 * device buffer (256-byte aligned) for the whole batch.
 * aaqaoa_expect_multi: gamma, beta host, G*p doubles (graph-major); energy
 * host, G doubles (fused aggregation). Synchronises the batch's stream.
 * aaqaoa_multi_info: graphs, how many run in the small-graph kernel, the
 * chosen number of parallel branches, kernel launches per evaluation.
 */
typedef struct aaqaoa_multi aaqaoa_multi;
typedef struct {
    int n;
    int num_edges;
    const int32_t *edges;
    int num_orbits;
    const int32_t *orbit_rep;
    const int32_t *orbit_weight;
    const int32_t *edge_orbit;  /* num_edges int32 or NULL */
} aaqaoa_graph_desc;

int aaqaoa_prepare_multi(int G, const aaqaoa_graph_desc *graphs, int p, unsigned flags, void *stream,
                         aaqaoa_multi **out);
int aaqaoa_multi_workspace_bytes(const aaqaoa_multi *multi, size_t *bytes);
int aaqaoa_multi_set_workspace(aaqaoa_multi *multi, void *device_ptr, size_t bytes);
int aaqaoa_expect_multi(aaqaoa_multi *multi, const double *gamma, const double *beta, int observable,
                        double *energy);
int aaqaoa_multi_info(const aaqaoa_multi *multi, int *G, int *small_graphs, int *branches,
                      int *launches_per_call);
void aaqaoa_destroy_multi(aaqaoa_multi *multi);

/*
 * aaqaoa_inject_fault -- test hook for the failure path of the tiled passes.
 * kind AAQAOA_FAULT_DROP_TILE: the next tiled pass that loads the statevector
 * leaves the first tile of one CTA unloaded, so that CTA's bounded wait
 * (about one second) runs out; the call returns AAQAOA_ERR_TIMEOUT, its
 * results are invalid, and the plan keeps working for later calls. Nothing
 * faults: the wait is the same bounded wait every pass uses. kind 0 clears a
 * pending fault. Plans with n <= the tile size have no tiled pass
 * (AAQAOA_ERR_UNSUPPORTED).
 */
#define AAQAOA_FAULT_DROP_TILE 1
int aaqaoa_inject_fault(aaqaoa_plan *plan, int kind);

/*
 * Qubits per pass (the "fusion depth" of the tiled mixer, Sec. 2's H_M applied
 * as one butterfly per qubit): a layer is a low pass over qubits 0..L-1 plus K
 * high passes sharing the other n - L qubits. plan4 = {L, K} of the forward
 * passes and {L, K} of the two-vector adjoint passes (all 0 for plans small
 * enough for the whole-circuit kernel).
 *
 * aaqaoa_get_pass_plan: plan4 (host, 4 ints) receives the current plan.
 * aaqaoa_set_pass_plan: 0 keeps the default for that entry (the fewest high
 *   passes; a two-register-stage low pass when they can take the rest).
 *   For complex64 plans the adjoint's low pass may span 14 qubits (bwd_low =
 *   14): a cluster of 4 CTAs loads the 2^14 contiguous amplitudes of a tile,
 *   a quarter each, and exchanges them through distributed shared memory so
 *   that the last two of the 14 qubits are mixed too; a layer then needs one
 *   high pass fewer (n = 30: 14 + 8 + 8 instead of 8 + 8 + 7 + 7). A batch of
 *   B points runs that pass once per point.
 *   INVALID_ARG if an (L, K) does not tile n with rows of >= 128 bytes.
 *   Rebuilds the workspace's tensor maps; the stored state becomes invalid.
 * aaqaoa_autotune: times each candidate (the fewest and one more high pass,
 *   each with the full and the two-stage low pass, and for the complex64
 *   adjoint the 14-qubit cluster low pass) on the plan's workspace
 *   and stream and keeps the fastest forward and adjoint plans; the choice is
 *   cached per process by (device, precision, n, p, batch, gradient, layer
 *   fusion). Leaves
 *   garbage in the workspace's vectors. AAQAOA_AUTOTUNE=0 in the environment
 *   keeps the default plan. plan4 (host, 4 ints, or NULL) receives the result.
 */
int aaqaoa_get_pass_plan(aaqaoa_plan *plan, int *plan4);
int aaqaoa_set_pass_plan(aaqaoa_plan *plan, int fwd_low, int fwd_high, int bwd_low, int bwd_high);
int aaqaoa_autotune(aaqaoa_plan *plan, int *plan4);

/*
 * Layer-boundary fusion (Eq. (1): consecutive layers U_M(beta_l) U_C(gamma_{l+1})
 * meet at a diagonal step). With p >= 2 and at least two high passes per
 * layer, the pass that ends layer l also applies the next layer's cost phase
 * (the inverse phase in the adjoint) and its mixer on the same qubits, so the
 * statevector is read and written once less per layer boundary. The same
 * setting enables the turnaround pass of gradient evaluations (the forward's
 * last pass and the adjoint's first in one launch, see aaqaoa_get_schedule;
 * any p >= 1). Results are the same up to rounding order. enable: 1 (the
 * default) or 0.
 * aaqaoa_get_layer_fusion writes the setting to *enable (host int).
 * INVALID_ARG for a NULL plan/pointer or enable not 0/1. The stored state
 * becomes invalid.
 */
int aaqaoa_set_layer_fusion(aaqaoa_plan *plan, int enable);
int aaqaoa_get_layer_fusion(aaqaoa_plan *plan, int *enable);

/*
 * aaqaoa_get_schedule -- the tiled passes one sweep launches, in order, as
 * 5 ints each (host, row-major [cap][5]): the pass's first qubit s, its
 * qubit count, the layer l whose mixer it applies there, the second layer of
 * a fused pass or -1, and the number of layer l's qubits mixed by earlier
 * passes. adjoint = 0: the forward sweep of an energy evaluation; 1: the
 * adjoint sweep of a gradient evaluation; 2: the forward sweep of a gradient
 * evaluation. Forward sweeps run layers 0..p-1, the adjoint p-1..0; within
 * a layer the low pass comes first, except the first layer of a complex64
 * forward sweep with two or more high passes, which starts on a high group
 * (the pass that generates the state), and a layer ends on a high pass.
 * With layer fusion, when the forward's last group is one of the adjoint's
 * high groups, a gradient evaluation joins the forward's last pass and the
 * adjoint's first into one turnaround pass: it is the adjoint sweep's first
 * row, its second layer equal to its layer (the last layer, mixed forward on
 * phi, then back on phi and lambda), and the gradient's forward sweep
 * (adjoint = 2) leaves that group of the last layer to it (its last row may
 * then be a low pass). *count (host int) receives the number of passes; at
 * most cap rows are written. Needs no device. Plans small enough for the
 * whole-circuit kernel have no tiled passes (*count = 0).
 * INVALID_ARG for NULL plan/count, cap < 0, steps NULL with cap > 0, or
 * adjoint not 0, 1 or 2.
 */
int aaqaoa_get_schedule(aaqaoa_plan *plan, int adjoint, int32_t *steps, int cap, int *count);

/*
 * aaqaoa_edge_orbits -- the edge classes behind H_red, computed on the host
 * (Sec. 4, Algorithm 1): generators of Aut(G) from an individualisation-
 * refinement search (each checked to map E onto E), then the breadth-first
 * closure of every unclassified edge, in the given edge order, under them.
 * No GPU is used.
 * n: 1..64 vertices. edges: 2*num_edges int32, unordered pairs, no loops or
 * repeats. edge_weight: num_edges int32 >= 1 (weighted MaxCut: only
 * automorphisms that keep every edge's weight count), or NULL for unweighted.
 * Outputs (host, caller-owned): edge_orbit[num_edges] class of each
 * edge; *num_orbits; orbit_rep[<= num_edges] the seed (lowest-index) edge of
 * each class; orbit_weight[<= num_edges] class sizes |S~_m|. These are
 * exactly the orbit arguments of aaqaoa_prepare.
 * Returns AAQAOA_ERR_INVALID_ARG for bad sizes, pointers or edges.
 */
int aaqaoa_edge_orbits(int n, int num_edges, const int32_t *edges, const int32_t *edge_weight, int32_t *edge_orbit,
                       int32_t *num_orbits, int32_t *orbit_rep, int32_t *orbit_weight);

/*
 * aaqaoa_ising_orbits -- edge and vertex classes for an Ising-form objective
 * (aaqaoa_prepare_ising): the same search and closure as aaqaoa_edge_orbits
 * over the automorphisms that keep every edge's real coupling (equal values)
 * and, when field is not NULL, every vertex's real field (Sec. 4 with the
 * couplings and fields as edge and vertex colours). No GPU is used.
 * n: 1..64. edges: 2*num_edges int32. edge_weight: num_edges doubles.
 * field: n doubles or NULL. Outputs (host, caller-owned): edge_orbit,
 * *num_orbits, orbit_rep, orbit_weight as for aaqaoa_edge_orbits;
 * vertex_orbit[n] class of each vertex, *num_vorbits, vorbit_rep[<= n] the
 * smallest vertex of each class, vorbit_weight[<= n] class sizes; classes are
 * numbered by smallest member. These are the orbit arguments of
 * aaqaoa_prepare_ising. Returns AAQAOA_ERR_INVALID_ARG for bad sizes,
 * pointers, edges, or a NaN weight or field.
 */
int aaqaoa_ising_orbits(int n, int num_edges, const int32_t *edges, const double *edge_weight, const double *field,
                        int32_t *edge_orbit, int32_t *num_orbits, int32_t *orbit_rep, int32_t *orbit_weight,
                        int32_t *vertex_orbit, int32_t *num_vorbits, int32_t *vorbit_rep, int32_t *vorbit_weight);

/* Plan properties: qubits, layers, edges, orbits, precision flag. */
int aaqaoa_plan_info(const aaqaoa_plan *plan, int *n, int *p, int *num_edges, int *num_orbits,
                     unsigned *flags);

/*
 * aaqaoa_launch_count -- number of kernel launches the last completed call on
 * this plan enqueued (for launch accounting in benchmarks).
 */
int aaqaoa_launch_count(const aaqaoa_plan *plan, int *launches);

/*
 * Launch profiling. While enabled, the plan records a CUDA event pair on its
 * stream around every kernel launch and keeps, per kernel kind, the launch
 * count and the bytes each launch has to move (statevector tiles loaded plus
 * stored). aaqaoa_profile_read synchronises the stream and returns the summed
 * event durations (ms), launches and bytes of one kind:
 *   0 forward tiled pass, 1 adjoint tiled pass, 2 whole-circuit (small n)
 *   kernel, 3 aggregation over a stored state, 4 parameter tables.
 * aaqaoa_profile_enable(plan, 0) stops recording; enabling clears the record.
 */
int aaqaoa_profile_enable(aaqaoa_plan *plan, int enable);
int aaqaoa_profile_read(aaqaoa_plan *plan, int kind, double *ms_total, int *launches, double *bytes);

/*
 * aaqaoa_stats -- all kinds of aaqaoa_profile_read at once: per kind (index
 * as above) the launches recorded since profiling was enabled, their summed
 * event durations (ms) and the bytes they had to move. out: host struct.
 * Synchronises the plan's stream (so the plan is not const). INVALID_ARG for
 * a NULL plan or out; all zero when profiling was never enabled.
 */
#define AAQAOA_STAT_KINDS 5
typedef struct {
    int launches[AAQAOA_STAT_KINDS];
    double ms[AAQAOA_STAT_KINDS];
    double bytes[AAQAOA_STAT_KINDS];
} aaqaoa_stats_t;
int aaqaoa_stats(aaqaoa_plan *plan, aaqaoa_stats_t *out);

/*
 * aaqaoa_profile_launches -- the recorded launches one by one, in launch
 * order: per launch its kind (as above), flags (bit 0: the pass carries
 * cut-function work -- phase, lambda = O phi, energy, dE/dgamma, inverse
 * phase; bit 1: a fused layer boundary; bit 2: the cluster low pass; bit 3:
 * the turnaround pass of a gradient evaluation), event duration (ms) and
 * bytes to move. kind, flags, ms, bytes: host arrays of at least max entries, each may
 * be NULL. *count (host int) receives the number of records, also when it
 * exceeds max. Synchronises the plan's stream. INVALID_ARG for a NULL plan
 * or count, or max < 0.
 */
int aaqaoa_profile_launches(aaqaoa_plan *plan, int max, int *count, int *kind, int *flags, double *ms,
                            double *bytes);

/* Release a plan (not the workspace, which the caller owns). NULL is a no-op. */
void aaqaoa_destroy(aaqaoa_plan *plan);

/* Fixed description of an error code. */
const char *aaqaoa_strerror(int code);

/* Message recorded by the last failing call on this thread ("" if none). */
const char *aaqaoa_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* AAQAOA_H */

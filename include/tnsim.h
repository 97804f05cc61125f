/*
 * tnsim.h -- C ABI of the GB300 (sm_103a) MPS two-qubit-gate library.
 *
 * The library applies layers of nearest-neighbour two-qubit gates to a Matrix
 * Product State held in GPU memory (HBM).  Per gate on the adjacent pair
 * (q, q+1) it runs the steps of the paper's local two-qubit update (Sec. III.A
 * "Two Qubit Gate", Sec. IV.A simulation_kernel, Fig. 2):
 *
 *   merge the two sites over their shared bond, contract the 4x4 gate (Eq. 1),
 *   take a truncated SVD of the (2 chi_L) x (2 chi_R) result, write the left
 *   singular vectors into site q and S.V^H into site q+1.
 *
 * All gates of a layer act on disjoint pairs and run in the same launches
 * (Sec. IV.B "Parallelizing the TAMM Backend": layers of non-overlapping gates).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Qubit 0 is the leftmost site and the most significant bit of a bitstring.
 *  - Site q is a tensor (chi_q, 2, chi_{q+1}), row-major, complex, with
 *    chi_0 = chi_n = 1 (Eq. 2).
 *  - A two-qubit gate is a 4x4 complex128 matrix, row-major, real and imaginary
 *    parts interleaved (32 doubles), basis index 2*b_q + b_{q+1}.
 *  - A one-qubit gate is a 2x2 complex128 matrix, row-major, interleaved (8 doubles).
 *  - Every function returns a tnsim_status and never throws or aborts across the
 *    ABI.  On failure tnsim_last_error() returns a thread-local message.
 *  - Host buffers passed in are read before the call returns; output host
 *    buffers are owned by the caller.  Device memory of a handle is allocated by
 *    the library (cudaMalloc) at tnsim_mps_create and freed by tnsim_mps_destroy.
 *  - Device-side failures (a Jacobi SVD that hit its sweep cap) set a status word
 *    in device memory; they never trap.  They are reported by the next
 *    synchronising call.
 */
#ifndef TNSIM_H
#define TNSIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tnsim_mps tnsim_mps; /* opaque handle */

typedef enum {
    TNSIM_OK = 0,
    TNSIM_EINVAL = 1,      /* bad argument; nothing was launched, the state is unchanged */
    TNSIM_ENOMEM = 2,      /* a device or pinned allocation failed */
    TNSIM_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error) */
    TNSIM_ENOCONV = 4,     /* a Jacobi SVD reached max_sweeps; the layer was still applied */
    TNSIM_ETIMEOUT = 5,    /* a bounded device wait ran out; the layer is incomplete (state undefined) */
    TNSIM_EUNSUPPORTED = 6 /* entry point or mode not available in this build */
} tnsim_status;

typedef enum { TNSIM_C64 = 0, TNSIM_C128 = 1 } tnsim_dtype;

/* How a layer is scheduled on the GPU. */
typedef enum {
    TNSIM_SCHED_BATCHED = 0, /* every pair of the layer in the same launches */
    TNSIM_SCHED_PLAIN = 1    /* one pair at a time (the per-pair comparison path) */
} tnsim_schedule;

/* Arithmetic of the merge + gate contraction for complex64 states (complex128 states
 * always use FP64 FMA).  The singular value decomposition is FP32 in every mode. */
typedef enum {
    TNSIM_GEMM_FP32 = 0,    /* FP32 FMA, four real products per complex product (4M) */
    TNSIM_GEMM_FP32_3M = 1, /* FP32 FMA, three real products per complex product (3M) */
    TNSIM_GEMM_TF32X3 = 2,  /* tensor cores (tcgen05 kind::tf32): 3 split TF32 products, FP32 accumulate */
    TNSIM_GEMM_BF16X3 = 3   /* tensor cores (tcgen05 kind::f16): 3 split BF16 products, FP32 accumulate */
} tnsim_gemm_mode;

/* Form of the state that a two-qubit update maintains. */
typedef enum {
    TNSIM_FORM_PAPER = 0,    /* the paper's update (Sec. III.A): U to the left site, S.V^H to the right */
    TNSIM_FORM_CANONICAL = 1 /* right-canonical sites with every bond's singular values kept beside them
                                (Hastings form): the SVD is of diag(Lam_q) theta, whose singular values are
                                the Schmidt coefficients of the cut, so truncation is optimal for the
                                state; the right site becomes V^H and the left site theta.V */
} tnsim_form;

typedef struct {
    int32_t chi_max;    /* bond-dimension cap, >= 1 (Sec. II.A: truncate to a fixed chi) */
    double cutoff;      /* relative discarded-weight cutoff in [0, 1); 0 = none */
    int32_t renormalize;/* 1: rescale kept singular values so sum s^2 is unchanged */
    int32_t max_sweeps; /* Jacobi sweep cap; 0 = default (40 c64, 60 c128) */
    double jacobi_tol;  /* rotate a column pair while |g| > tol*sqrt(a*b); 0 = default
                           (complex64: 2 eps_32; complex128: max(sqrt(2 chi_L), 4) eps_64) */
    int32_t schedule;   /* tnsim_schedule */
    int32_t gemm;       /* tnsim_gemm_mode (complex64 only) */
    int32_t form;       /* tnsim_form */
} tnsim_params;

/* Fill *out with the defaults for dtype dt (chi_max 64, cutoff 0, renormalize 1,
 * batched schedule, FP32 contraction, the paper's form).
 * Errors: EINVAL if out is NULL or dt unknown. */
tnsim_status tnsim_params_default(tnsim_dtype dt, tnsim_params* out);

/* Create the state |0...0> on n_qubits >= 2 sites with every bond of dimension 1
 * (Sec. IV.A "Implementations").  dt selects complex64 (FP32 arithmetic) or
 * complex128 (FP64 arithmetic).  p may be NULL (defaults).  cuda_stream is a
 * cudaStream_t on which all work of this handle is ordered; NULL makes the
 * library create and own a non-blocking stream.  Device memory for the sites
 * (capacity min(2^q, 2^(n-q), chi_max) per bond) and for one layer's workspace
 * is allocated here on the current device.
 * Errors: EINVAL (n_qubits < 2, bad params), ENOMEM, ECUDA. */
tnsim_status tnsim_mps_create(int32_t n_qubits, tnsim_dtype dt, const tnsim_params* p,
                              void* cuda_stream, tnsim_mps** out);

/* Release every device and host resource of m (NULL is accepted). Synchronises m's stream. */
tnsim_status tnsim_mps_destroy(tnsim_mps* m);

/* Apply one layer (Sec. III.A "One Qubit Gate" / "Two Qubit Gate", Sec. IV.B layers):
 *   u1  : NULL, or n_qubits one-qubit gates (8 doubles each) applied to every qubit
 *         BEFORE the two-qubit gates (identity entries are allowed);
 *   q   : n2 left-qubit indices; the pairs (q[i], q[i]+1) must be disjoint;
 *   g4x4: n2 two-qubit gates (32 doubles each), host memory.
 * eps_out (may be NULL) receives the relative discarded weight of each gate,
 * sum_{j>=k} s_j^2 / sum_j s_j^2.  The call is synchronous: it returns after the
 * layer finished on the GPU.  Errors: EINVAL (bad pair list, non-finite gate,
 * n2 < 0; nothing launched), ENOCONV (layer applied, an SVD hit max_sweeps),
 * ETIMEOUT (a bounded device wait ran out, see tnsim_set_wait_limits), ECUDA. */
tnsim_status tnsim_apply_layer(tnsim_mps* m, int32_t n2, const int32_t* q,
                               const double* g4x4, const double* u1, double* eps_out);

/* Same layer with the gate data already in device memory: g4x4_dev (n2*32 doubles),
 * u1_dev (n_qubits*8 doubles or NULL); q stays a host array.  eps_dev (device,
 * n2 doubles, may be NULL) receives the discarded weights.  Asynchronous: work is
 * only ordered on the handle's stream; device-side status is collected by
 * tnsim_sync.  Errors: EINVAL (bad pair list; nothing launched), ECUDA. */
tnsim_status tnsim_apply_layer_device(tnsim_mps* m, int32_t n2, const int32_t* q,
                                      const double* g4x4_dev, const double* u1_dev,
                                      double* eps_dev);

/* Apply a list of gates on any qubits (Sec. IV.B: non-local two-qubit gates by the
 * SWAP method, and layerization into non-overlapping layers).
 *   operation i : qb[i] < 0 -- a one-qubit gate on qubit qa[i], 2x2 in the first 8
 *                 doubles of mats[32*i ...];
 *                 qb[i] >= 0 -- a two-qubit gate on the distinct qubits qa[i], qb[i]
 *                 (any distance, either order), 4x4 in mats[32*i ...] with basis
 *                 index 2*b_qa + b_qb.
 * A gate on qubits lo < hi with hi - lo > 1 runs as: SWAP(hi-1, hi), ...,
 * SWAP(lo+1, lo+2), the gate on (lo, lo+1), then the same SWAPs in reverse order;
 * each SWAP is an ordinary truncating two-qubit update.  The local operations are
 * cut into layers as soon as possible (one-qubit gates share a layer with the
 * next two-qubit gate on their qubit), which gives the same state as applying the
 * list in order.  n_layers_out / n_gates_out (may be NULL) receive the number of
 * layers and of local two-qubit updates (SWAPs included); eps_sum_out (may be
 * NULL) the sum of their discarded weights.  The gate data is copied to the device
 * once (a stream-ordered allocation freed at the end); the layers are launched back
 * to back without host synchronisation; the call synchronises at the end.
 * Errors: EINVAL (bad qubit, equal qubits, non-finite entry; nothing launched),
 * ENOCONV (applied; an SVD hit max_sweeps), ETIMEOUT (state undefined), ECUDA. */
tnsim_status tnsim_apply_circuit(tnsim_mps* m, int32_t n_ops, const int32_t* qa, const int32_t* qb,
                                 const double* mats, int32_t* n_layers_out, int32_t* n_gates_out,
                                 double* eps_sum_out);

/* The host planner of tnsim_apply_circuit on its own (no GPU work, no handle):
 * expand the same operation list (n_qubits qubits) into layers.  n_layers and
 * n_gates (required) receive the sizes.  If layer_n2, gate_q, gate_g4 and layer_u1
 * are all NULL only the sizes are computed; otherwise every one must be given with
 * cap_layers >= *n_layers and cap_gates >= *n_gates:
 *   layer_n2 [n_layers]        pairs per layer;
 *   gate_q   [n_gates]         left qubit of each pair, layer after layer;
 *   gate_g4  [n_gates * 32]    the 4x4 of each pair (basis 2*b_q + b_{q+1});
 *   layer_u1 [n_layers * n_qubits * 8]  the one-qubit gates of each layer, applied
 *                              before its pairs (identity where none).
 * Errors: EINVAL (bad operation, capacity too small). */
tnsim_status tnsim_circuit_layerize(int32_t n_qubits, int32_t n_ops, const int32_t* qa, const int32_t* qb,
                                    const double* mats, int32_t cap_layers, int32_t cap_gates,
                                    int32_t* n_layers, int32_t* n_gates, int32_t* layer_n2,
                                    int32_t* gate_q, double* gate_g4, double* layer_u1);

/* Apply layers to several independent states in one batched schedule: for each
 * step t in [0, n_steps), state ms[i] gets the layer described by
 * (n2[t*n_circ+i], q_ptrs[...], g_ptrs[...], u1_ptrs[...]) -- all host arrays in
 * the same formats as tnsim_apply_layer (a NULL u1 pointer means no 1q gates;
 * n2 = 0 and no u1 means the state skips that step).  All states must share the
 * dtype.  Every step's pairs of every state run in the same launches.  Synchronous.
 * Errors: EINVAL, ENOCONV, ECUDA. */
tnsim_status tnsim_apply_layers_batched(tnsim_mps* const* ms, int32_t n_circ, int32_t n_steps,
                                        const int32_t* n2, const int32_t* const* q_ptrs,
                                        const double* const* g_ptrs,
                                        const double* const* u1_ptrs);

/* A frozen layer: the descriptors, workspace and launch shapes of one layer of one or
 * more states, built once so that replaying it needs no host work.  Gate data is read
 * at replay from the device buffers given here (g4_dev[i]: n2[i]*32 doubles, u1_dev[i]:
 * n_qubits*8 doubles or NULL), so a caller can refresh their contents between
 * replays.  Grid shapes are sized for the states' bond capacities, so a plan stays
 * valid however the bonds grow.  All states must share dtype, device, stream and gemm
 * mode.  Synchronous (uploads the descriptors).  Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct tnsim_plan tnsim_plan;
tnsim_status tnsim_plan_create(tnsim_mps* const* ms, int32_t n_states, const int32_t* n2,
                               const int32_t* const* q_ptrs, const double* const* g4_dev,
                               const double* const* u1_dev, tnsim_plan** out);

/* Enqueue a plan's kernels and memsets on the first state's stream (no host
 * synchronisation, no host copies: it can be captured into a CUDA graph).  The
 * discarded weights are not returned; tnsim_sync collects the status. */
tnsim_status tnsim_plan_launch(tnsim_plan* plan);
tnsim_status tnsim_plan_destroy(tnsim_plan* plan);

/* A CUDA graph holding the launches of n_plans plans in order (captured on the first
 * plan's stream in relaxed mode), replayed by tnsim_graph_launch on that stream.
 * Errors: EINVAL, ECUDA. */
typedef struct tnsim_graph tnsim_graph;
tnsim_status tnsim_graph_create(tnsim_plan* const* plans, int32_t n_plans, tnsim_graph** out);
tnsim_status tnsim_graph_launch(tnsim_graph* g);
tnsim_status tnsim_graph_destroy(tnsim_graph* g);

/* Wait for the handle's stream and return the sticky device status (OK or ENOCONV),
 * clearing it.  Errors: ECUDA. */
tnsim_status tnsim_sync(tnsim_mps* m);

/* Current bond dimensions chi_0..chi_n (n_qubits+1 int32, host).  Synchronises. */
tnsim_status tnsim_bond_dims(tnsim_mps* m, int32_t* out);

/* Singular values kept on bond b (between sites b-1 and b) by the last SVD that
 * wrote it, after renormalisation; s_out holds chi_max doubles (host), *k_out the
 * count (0 if no SVD has written that bond).  Synchronises.  Errors: EINVAL. */
tnsim_status tnsim_bond_spectrum(tnsim_mps* m, int32_t bond, double* s_out, int32_t* k_out);

/* Copy every site to host as complex128 interleaved, site after site, each
 * (chi_q, 2, chi_{q+1}) row-major.  cap is the number of doubles out can hold;
 * *needed (may be NULL) receives the number required.  Synchronises.
 * Errors: EINVAL if cap is too small (nothing written). */
tnsim_status tnsim_export_sites(tnsim_mps* m, double* out, int64_t cap, int64_t* needed);

/* Replace the state by host sites in the export layout; dims holds chi_0..chi_n
 * (chi_0 = chi_n = 1, chi_q within the handle's capacity).  The stored bond spectra
 * are cleared.  Synchronous.
 * Errors: EINVAL (dims out of range), EUNSUPPORTED (a TNSIM_FORM_CANONICAL state: its
 * bond spectra would be unknown). */
tnsim_status tnsim_import_sites(tnsim_mps* m, const int32_t* dims, const double* data);

/* <x|psi> for n_str bitstrings (bits: n_str*n_qubits bytes of 0/1, host, qubit 0
 * first) -- Eq. 2 with every physical leg fixed.  amps_out: n_str complex128
 * interleaved (host).  Synchronous.  Errors: EINVAL. */
tnsim_status tnsim_amplitudes(tnsim_mps* m, int64_t n_str, const uint8_t* bits,
                              double* amps_out);

/* <psi| P |psi> for n_terms Pauli strings (paulis: n_terms*n_qubits chars from
 * 'I','X','Y','Z', host).  out: n_terms complex128 interleaved (host).  The state
 * is not normalised first.  Synchronous.  Errors: EINVAL (bad character). */
tnsim_status tnsim_expect_pauli(tnsim_mps* m, int32_t n_terms, const char* paulis,
                                double* out);

/* Perfect sampling of n_shots bitstrings (Sec. III.A "Sampling"; Sec. IV.A
 * measurement).  Qubit by qubit from qubit 0, shot s takes bit b_q = 1 exactly when
 * uniforms[s*n + q] * (p0 + p1) >= p0, where p0, p1 are the weights of the two
 * outcomes given its earlier bits; the prefix is then projected on the outcome
 * and renormalised.  The weights use the right environments of the state, which
 * gives the same numbers as sampling its right-canonical form.  Shots with the
 * same prefix share its vector (memoised prefixes): each site evaluates only the
 * distinct prefixes.
 *   uniforms : host, n_shots * n_qubits doubles in [0, 1), row s = shot s;
 *   bits_out : host, n_shots * n_qubits bytes (0/1), qubit 0 first;
 *   n_nodes_out (may be NULL): distinct prefixes evaluated, summed over the sites.
 * Work buffers come from one stream-ordered allocation freed at the end.
 * Synchronous.  Errors: EINVAL (n_shots outside [0, 2^24], NULL, a uniform outside
 * [0, 1)), ECUDA. */
tnsim_status tnsim_sample(tnsim_mps* m, int64_t n_shots, const double* uniforms, uint8_t* bits_out,
                          int64_t* n_nodes_out);

/* Launch configurations of the Jacobi SVD.  Bit 0: 0 -- 16-column blocks (8 for
 * complex128 at chi > 128), one persistent CTA per SM; 1 -- half-width blocks, two
 * CTAs per SM (barriers of the two CTAs are independent; a sweep has twice the
 * rounds).  Bit 1: QR preconditioning (Drmac and Veselic 2008) of every gate whose
 * gated block is square (2 chi_L == 2 chi_R <= 1536) in the paper's form: theta = Q R
 * by blocked Householder reflections, the Jacobi iteration runs on the columns of
 * R^H (fewer sweeps), the left site is theta V S^-1 and the right site S V^H is read
 * off the converged columns; Q is never formed.  Bit 2 (complex64 states): every
 * visit forms the block pair's Gram matrix X^H X on the tensor cores, applies the
 * visit's rotations to it (same order and parameters as the column rotations) while
 * accumulating the rotation V, and updates the columns as X V on the tensor cores
 * (3xTF32); bit 0 then has no effect, and complex128 states run bits 0-1 only.  Same
 * kept spectrum and state up to the Jacobi tolerance in every configuration. */
#define TNSIM_JACOBI_CONFIGS 8

/* Use Jacobi configuration cfg (0 .. TNSIM_JACOBI_CONFIGS - 1) for the later
 * launches of m.  Errors: EINVAL. */
tnsim_status tnsim_set_jacobi_config(tnsim_mps* m, int32_t cfg);

/* Limits of the two bounded waits inside the layer kernels (no kernel traps or waits
 * forever; a wait that runs out is reported through the gate's status word).  The paper
 * has no counterpart: it is the failure handling of this library's persistent launch.
 *   jacobi_idle_polls : polls (each followed by a short sleep) an idle CTA of the
 *                       persistent Jacobi launch makes without seeing any gate's round
 *                       complete before it sets the launch's error flag; every CTA then
 *                       leaves, the unfinished gates report status 5;
 *   mbarrier_polls    : polls of one mbarrier wait (TMA copies landed, MMAs done) in the
 *                       tensor-core kernels (the contraction, the Gram-matrix Jacobi visits
 *                       of configurations 4-7, the left site of the QR configurations); on
 *                       timeout the CTA waits (with the default limit) for the copies or
 *                       MMAs it already issued, then leaves and reports status 5 for its
 *                       gate.
 * 0 restores a default (2^22 and 2^26 polls: about a second or more, far beyond any
 * legitimate wait).
 * Calls after a timeout return ETIMEOUT; the state is undefined but the handle and
 * the CUDA context stay usable (import sites or start again).
 * Errors: EINVAL (NULL state, negative limit or one beyond 32 bits). */
tnsim_status tnsim_set_wait_limits(tnsim_mps* m, int64_t jacobi_idle_polls, int64_t mbarrier_polls);

/* Process-wide cap on the device memory held by the states of this library (0 = no cap,
 * the default).  tnsim_mps_create computes every device allocation of the new state
 * before making any, and returns ENOMEM, allocating nothing, when the bytes already held
 * plus the new state's would exceed the cap.  Errors: EINVAL (negative bytes). */
tnsim_status tnsim_set_device_memory_cap(int64_t bytes);

/* Device bytes held by the live states of this process (as counted for the cap). */
int64_t tnsim_device_bytes_held(void);

/* Autotuner of the Jacobi SVD: contract the given layer (n2 >= 1 pairs q, gates
 * g4x4 on the host, as in tnsim_apply_layer) of the current state into the work
 * space, then time the persistent Jacobi launch of that layer in every
 * configuration (CUDA events on m's stream, the QR factorisation included where
 * the configuration has it; W and the gate records are restored before each
 * launch; the best of reps runs is kept), pick the fastest for m's
 * later launches and report it in *choice_out (may be NULL); ms_out (may be NULL)
 * receives TNSIM_JACOBI_CONFIGS times in milliseconds.  The state is not changed.
 * Synchronous.  Errors: EINVAL (bad layer, reps outside [1, 100]), ECUDA. */
tnsim_status tnsim_autotune(tnsim_mps* m, int32_t n2, const int32_t* q, const double* g4x4, int32_t reps,
                            int32_t* choice_out, double* ms_out);

/* A layered circuit for tnsim_grad.  Layer L: every qubit gets n_rot[L] rotations
 * R_a(t) = exp(-i t P_a / 2) (axes: the n_rot[L] letters 'X','Y','Z' of the layer,
 * concatenated over layers; the first letter acts first), then n2[L] fixed two-qubit
 * gates on disjoint pairs (q[...], q[...]+1), 4x4 in g4x4 (32 doubles each), both
 * concatenated over layers.  The angles theta are laid out layer after layer as
 * [n_qubits][n_rot[L]]. */
typedef struct {
    int32_t n_qubits;
    int32_t n_layers;
    const int32_t* n_rot;
    const char* axes;
    const int32_t* n2;
    const int32_t* q;
    const double* g4x4;
} tnsim_circuit;

/* H = sum_t coeffs[t] P_t: n_terms Pauli strings of n_qubits letters from 'I','X','Y','Z'. */
typedef struct {
    int32_t n_terms;
    const char* paulis;
    const double* coeffs;
} tnsim_hamiltonian;

/* Energy E = <psi|H|psi> / <psi|psi> of the circuit's state from |0...0> and its
 * gradient with respect to every angle, by reverse-mode differentiation of the
 * simulation itself (the paper does not differentiate its simulator).  The forward
 * is the library's layer path (dtype dt, params p: chi_max, cutoff, renormalize;
 * the paper's form only), with the state checkpointed before every layer.  The
 * backward starts from the adjoint of the final sites (transfer-matrix environments
 * of every Pauli term) and, layer by layer in reverse, restores the checkpoint,
 * recomputes the layer and differentiates each two-qubit update exactly: the new
 * left site U depends on the gated block T only through the kept subspace, whose
 * derivative couples kept and discarded singular directions through broadened
 * 1/(s_j^2 - s_l^2); the renormalisation factor is differentiated too.  So the
 * gradient is that of the truncated simulation.  cuda_stream: as in
 * tnsim_mps_create.  energy_out: host double; grad_out: host, sum_L n_qubits *
 * n_rot[L] doubles.  Synchronous; all device memory is released before return.
 * Errors: EINVAL (bad circuit, angles or Hamiltonian), EUNSUPPORTED (canonical
 * form), ENOMEM, ETIMEOUT, ECUDA. */
tnsim_status tnsim_grad(const tnsim_circuit* c, const double* theta, const tnsim_hamiltonian* h, tnsim_dtype dt,
                        const tnsim_params* p, void* cuda_stream, double* energy_out, double* grad_out);

/* Work counters accumulated on the device since the previous tnsim_last_stats call
 * on m (then reset).  visit_rows and rotation_rows weight every examined / rotated
 * column pair by its column length m = 2 chi_L, so the Jacobi SVD's arithmetic is
 * 8 visit_rows + 20 rotation_rows real flops (FMA = 2): an examined pair forms
 * g = x_i^H x_j, the column norms being tracked, and a rotation updates both columns. */
typedef struct {
    int64_t gates;         /* two-qubit gates applied */
    int64_t sweeps;        /* Jacobi sweeps, summed over gates */
    int64_t rotations;     /* column-pair rotations applied */
    int64_t pair_visits;   /* column pairs examined */
    int64_t visit_rows;    /* sum over examined pairs of m */
    int64_t rotation_rows; /* sum over rotated pairs of m */
    int64_t theta_cmacs;   /* complex multiply-adds of the merge (2chi_L chi_M 2chi_R per gate) */
    int64_t right_cmacs;   /* complex multiply-adds of the site product: the right site
                              (k 2chi_L 2chi_R per gate), or with QR preconditioning the
                              left site (same count) */
    int64_t qr_cmacs;      /* complex multiply-adds of the QR preconditioning, Householder's
                              count 2 n^3 / 3 per preconditioned n x n gate block */
} tnsim_stats;

/* Read (and reset) the counters.  Synchronises.  Errors: EINVAL. */
tnsim_status tnsim_last_stats(tnsim_mps* m, tnsim_stats* out);

/* Kernel classes timed by the optional profiler, in launch order within a layer. */
enum { TNSIM_K_SITE1Q = 0, TNSIM_K_THETA = 1, TNSIM_K_JACOBI = 2, TNSIM_K_TRUNCATE = 3,
       TNSIM_K_LEFT = 4, TNSIM_K_RIGHT = 5, TNSIM_K_QR = 6, TNSIM_K_COUNT = 7 };

/* Enable (on != 0) or disable per-kernel timing: while enabled every layer records
 * CUDA events on the handle's stream around each of its kernel launches (no extra
 * synchronisation).  Disabling drops unread records.  Errors: ECUDA. */
tnsim_status tnsim_profile_enable(tnsim_mps* m, int32_t on);

/* Sum of the device durations (milliseconds) of every recorded launch per kernel
 * class since the last read, and the number of launches per class; both arrays
 * have TNSIM_K_COUNT entries.  Synchronises, then resets.  Errors: EINVAL, ECUDA. */
tnsim_status tnsim_profile_read(tnsim_mps* m, double* ms, int64_t* launches);

/* One two-qubit update (merge, gate, truncated SVD, absorption; complex64) that
 * allocates no memory.  The paper has no counterpart: it is for callers that cannot
 * let a library call cudaMalloc -- a plugin inside an application whose memory pool
 * owns the whole device, a process under a fixed device-memory budget, or a loop
 * that must not synchronise the device (cudaMalloc/cudaFree may).
 *   site_a  : device, complex64 (chi_l, 2, chi_m) row-major, overwritten by the new
 *             left site (chi_l, 2, k); cap_a = its capacity in complex elements,
 *             >= chi_l * 2 * max(chi_m, kmax) with kmax = min(chi_max, 2chi_l, 2chi_r);
 *   site_b  : device, complex64 (chi_m, 2, chi_r), overwritten by the new right site
 *             (k, 2, chi_r); cap_b >= max(chi_m, kmax) * 2 * chi_r;
 *   g4x4    : host, the 4x4 complex128 gate (32 doubles); chi_max, cutoff and
 *             renormalize as in tnsim_params;
 *   cuda_stream : the cudaStream_t to run on (NULL = the legacy default stream);
 *   k_out   : host, the kept bond dimension; eps_out (host, may be NULL) the
 *             discarded weight; s_out (host, may be NULL, chi_max doubles) the kept
 *             singular values in its first k entries (the rest set to 0).
 * Limits: chi_l, chi_r <= 128 and chi_max <= 256 (EINVAL beyond).  Scratch is one
 * fixed array of about 1.1 MB compiled into the library, held by every GPU that
 * loads it until the process exits.  The first call on a device looks up that
 * array's device address; make that first call before any stream capture.  All
 * calls share the array, so calls whose work overlaps on the GPU race.  Synchronous.
 * Errors: EINVAL, ENOCONV (the update was applied), ETIMEOUT (the Jacobi kernel gave up
 * waiting; the sites are undefined), ECUDA, EUNSUPPORTED. */
tnsim_status tnsim_two_site_update_noalloc(void* site_a, int64_t cap_a, void* site_b,
                                           int64_t cap_b, int32_t chi_l, int32_t chi_m,
                                           int32_t chi_r, const double* g4x4, int32_t chi_max,
                                           double cutoff, int32_t renormalize, void* cuda_stream,
                                           int32_t* k_out, double* eps_out, double* s_out);

/* Thread-local description of the last failure (empty string if none). */
const char* tnsim_last_error(void);

/* Library version string. */
const char* tnsim_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TNSIM_H */

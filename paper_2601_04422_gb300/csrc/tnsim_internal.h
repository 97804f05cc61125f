// Internal declarations shared by the kernels and the C-ABI host runtime.
// Nothing here is part of the public ABI (include/tnsim.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tnsim {

// complex element type per arithmetic precision: interleaved (re, im)
template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };

// Results of one two-qubit update, written by the kernels (device memory).
struct GateOut {
    double frob2;                  // |theta|_F^2, accumulated by the theta kernel (FP64)
    double eps;                    // relative discarded weight sum_{j>=k} s_j^2 / sum_j s_j^2
    double scale;                  // renormalisation factor applied to the kept s
    int k;                         // kept bond dimension
    int sweeps;                    // Jacobi sweeps run (the last one rotated nothing if converged)
    int status;                    // 0 ok, 4 = the Jacobi SVD reached its sweep cap
    int finished;                  // the Jacobi iteration of this gate has ended
    int done;                      // visits of the current round reported
    int rot_sweep;                 // rotations of the current sweep
    unsigned long long claim;      // (round << 32) | visits of that round claimed
    unsigned long long rotations;  // column-pair rotations applied
    unsigned long long visits;     // column pairs examined
};

// Control word of one persistent Jacobi launch (zeroed before the launch).
struct JacobiCtl {
    int n_finished;                // gates whose iteration has ended
    int error;                     // set when idle CTAs saw no progress for too long
    unsigned int progress;         // rounds completed, over all gates
    int pad_;
};

// Everything a kernel needs about one gate (device memory, one per gate of a launch).
// Bond dimensions are read from chi[] at run time, so a launch can be issued
// before the previous layer's truncation ranks are known on the host.
struct GateDesc {
    void* siteA;          // slot of site q     (chi_q, 2, chi_{q+1}) row-major
    void* siteB;          // slot of site q+1   (chi_{q+1}, 2, chi_{q+2}) row-major
    int* chi;             // the state's bond dimensions chi_0..chi_n (device)
    const double* g4;     // 4x4 complex128 gate, row-major interleaved
    const double* uL;     // 2x2 complex128 applied to qubit q before g4, or null
    const double* uR;     // 2x2 complex128 applied to qubit q+1 before g4, or null
    void* theta0;         // (2chi_L) x (2chi_R) column-major copy of theta
    void* W;              // (2chi_L) x (2chi_R) column-major Jacobi working matrix
    double* s2;           // sorted squared column norms (length 2chi_R)
    int* perm;            // column index of each sorted entry
    double* spectrum;     // kept singular values of bond q+1 (chi_max doubles)
    int* spec_k;          // kept count of bond q+1
    double* eps_out;      // optional copy of the discarded weight (device), or null
    GateOut* out;
    int* sticky;          // the state's sticky status word (OR of gate statuses)
    unsigned long long* stats;  // the state's work counters (layout of tnsim_stats; the last one, qr_cmacs,
                                // only for QR-preconditioned gates)
    // split operand planes for the tensor-core contraction (complex64, TF32X3 / BF16X3)
    void* tc_planes;      // this state's plane buffer [slots * 8][tc_rows][tc_k]
    const void* tc_map_a; // CUtensorMap over the planes, 128-row boxes (device memory)
    const void* tc_map_b; // CUtensorMap over the planes, 64-row boxes (device memory)
    double cutoff;
    int q;
    int chi_max;
    int renorm;
    int tc_slot;          // this gate's slot in the plane buffer
    int tc_rows;          // rows of every plane (2 * capmax)
    int tc_k;             // K stride of every plane (capmax rounded up to 64)
    // canonical (Hastings) form: the SVD operand is diag(Lam_q) theta, the right site
    // becomes V^H and the left site theta V (k_canon.cu); 0 = the paper's form
    int canon;
    const double* lam;    // singular values of bond q (the state's spectrum of bond q)
    const int* lam_k;     // their count (0 = bond never decomposed: all ones)
    // QR preconditioning (k_qr.cu): for m == n the Jacobi runs on R^H of theta = Q R; the
    // left site becomes theta W' S^-2 and the right site the conjugated Jacobi columns
    int qr;
    // polls of a bounded mbarrier wait in the tensor-core contraction before it gives up
    // (0 = the kernel's default); the CTA then drains its copies in flight and reports
    // status 5 (ETIMEOUT)
    int wait_polls;
};

#ifdef __CUDACC__
// x^2 added to the double-length sum (s, c) with FP32 operations only: the product is
// split exactly (p + e = x^2 with e = fma(x, x, -p)) and p enters by Knuth's TwoSum, so
// s + c carries the sum to about eps^2 relative.  GB300 runs FP64 at 1/64 of the FP32
// rate; per-element FP64 arithmetic bounded the passes that accumulate norms.
__device__ __forceinline__ void add_sq(float x, float& s, float& c) {
    const float p = x * x;
    const float e = fmaf(x, x, -p);
    const float t = s + p;
    const float z = t - s;
    c += (s - (t - z)) + (p - z) + e;
    s = t;
}
// Sum of squares per thread: double-length FP32 for complex64, FP64 for complex128;
// value() is the FP64 result that the warp and block reductions combine.
template <typename T> struct SqAcc;
template <> struct SqAcc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) { add_sq(x, s, c); }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};
template <> struct SqAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s = fma(x, x, s); }
    __device__ __forceinline__ double value() const { return s; }
};
#endif

// largest m of a QR-preconditioned gate (its panel of columns sits in shared memory)
constexpr int kQrMaxRows = 1536;
#ifdef __CUDACC__
__device__ __forceinline__ bool qr_active(const GateDesc& d, int m, int n) {
    return d.qr && !d.canon && m == n && m <= kQrMaxRows;
}
#endif

// One-qubit update of one site (Eq. 3).
struct Site1Desc {
    void* site;
    const int* chi;
    const double* u;      // 2x2 complex128
    int q;
    int pad_;
};

// Launch wrappers (each returns the launch error, if any).
template <typename T>
cudaError_t launch_theta(const GateDesc* d, int n_gates, int chiL_max, int chiR_max,
                         cudaStream_t s);
// cfg bit 0 selects the block width / CTAs per SM (0: wide blocks, 1 CTA per SM; 1:
// half-width blocks, 2 CTAs per SM); bit 2 (complex64 only) the Gram-matrix visits with
// tensor-core block products (k_jacobi_tc.cu; bit 0 then has no effect).  Bit 1 of a
// state's configuration adds QR preconditioning (GateDesc::qr): kJacobiConfigs of them.
constexpr int kJacobiConfigs = 8;
// n_lead: how many leading descriptors (sorted by decreasing size) share the first one's
// size; the persistent CTAs start spread over them (0: over all gates).
// spin_limit: idle polls without progress before an idle CTA gives up (0 = default).
template <typename T>
cudaError_t launch_jacobi(const GateDesc* d, int n_gates, int m_max, int n_max, double tol,
                          int max_sweeps, JacobiCtl* ctl, cudaStream_t s, int cfg = 0, int n_lead = 0,
                          unsigned spin_limit = 0);
// the tensor-core Jacobi launch (complex64), called by launch_jacobi<float> for cfg bit 2
cudaError_t launch_jacobi_tc(const GateDesc* d, int n_gates, int n_lead, int n_max, double tol, int max_sweeps,
                             JacobiCtl* ctl, cudaStream_t s, unsigned spin_limit);
// the largest m (= 2 chi_L) the tensor-core Jacobi launch takes; larger gates run k_jacobi
int jacobi_tc_max_rows();
// n_max: the largest 2 chi_R of the batch (grid of the column-norm pass)
template <typename T>
cudaError_t launch_truncate(const GateDesc* d, int n_gates, int n_max, cudaStream_t s);
template <typename T>
cudaError_t launch_left(const GateDesc* d, int n_gates, int m_max, int k_max, cudaStream_t s);
template <typename T>
cudaError_t launch_right(const GateDesc* d, int n_gates, int k_max, int n_max, cudaStream_t s);
// Canonical form: scale W's rows by Lam_q (and recompute |W|_F^2); re-orthonormalise the
// new right site's rows and form the left site theta V.
template <typename T>
cudaError_t launch_scale_rows(const GateDesc* d, int n_gates, cudaStream_t s);
template <typename T>
cudaError_t launch_left_canon(const GateDesc* d, int n_gates, int m_max, int k_max, cudaStream_t s);
// QR preconditioning: W <- R^H of theta = Q R for every gate with qr_active; after the
// truncation, the left and right sites of those gates from the Jacobi columns
template <typename T>
cudaError_t launch_qr(const GateDesc* d, int n_gates, int m_max, cudaStream_t s);
template <typename T>
cudaError_t launch_sites_pre(const GateDesc* d, int n_gates, int m_max, int k_max, int n_max, cudaStream_t s,
                             int tc = 0);
// the left site of the QR-preconditioned complex64 gates on the tensor cores (3xTF32)
cudaError_t launch_left_pre_tc(const GateDesc* d, int n_gates, int m_max, int k_max, cudaStream_t s);
template <typename T>
cudaError_t launch_site1q(const Site1Desc* d, int n_sites, int cap_lr, cudaStream_t s);

// read-out
template <typename T>
cudaError_t launch_amplitudes(void* const* sites, const int* chi, int n_qubits, int chi_cap,
                              const uint8_t* bits, int64_t n_str, double* amps,
                              cudaStream_t s);
template <typename T>
cudaError_t launch_transfer(const void* site, const int* chi, int q, const double* op,
                            const void* e_in, void* tmp, void* e_out, int chi_cap,
                            int from_left, cudaStream_t s);
template <typename T>
cudaError_t launch_close(const void* E, const void* Rt, const int* chi, int bond, double* out,
                         cudaStream_t s);

// Merge + gate contraction with FP32 3M arithmetic (SIMT).
cudaError_t launch_theta_3m(const GateDesc* d, int n_gates, int chiL_max, int chiR_max, cudaStream_t s);
// Tensor-core merge + gate contraction (mode 0: 3xTF32, mode 1: BF16x3), split pass included.
cudaError_t launch_theta_tc(int mode, const GateDesc* d, int n_gates, int chiL_max, int chiM_max, int chiR_max,
                            cudaStream_t s);
// Encode the two tensor maps (opaque 128-byte CUtensorMap values) over a plane buffer.
cudaError_t encode_plane_maps(int mode, void* planes, int slots, int rows, int kstride, struct CUtensorMap_st* host_a,
                              struct CUtensorMap_st* host_b);

// Work buffers of perfect sampling (k_sample.cu); node arrays hold at most `shots` entries
struct SampleWork {
    void* v_cur;                   // [nodes][chi_max] prefix row vectors of this site
    void* v_next;                  // [nodes][chi_max] those of the next site
    void* w;                       // [nodes][2 chi_max]  v A_q
    void* y;                       // [2 nodes][chi_max]  (v A_q^b) Rt_{q+1}
    double* p;                     // [2 nodes] outcome weights
    int* flag;                     // [2 nodes] child (node, bit) drawn by some shot
    int* id;                       // [2 nodes] next-site index of each child, -1 if none
    int* parent;                   // [shots] child (2 node + bit) of each next-site node
    int* node_of;                  // [shots] node of each shot
    int* nodes;                    // current node count (device)
    unsigned long long* total;     // nodes summed over sites (device)
};
// One site of perfect sampling: weights, draws, memoised prefix update.  node_bound
// is a host upper bound of the current node count (min(shots, 2^q)).
template <typename T>
cudaError_t launch_sample_site(const void* site, int cl, int cr, const void* rt_next, int q, int n,
                               int64_t shots, int node_bound, const double* u, uint8_t* bits,
                               SampleWork& w, cudaStream_t s);

// ---------------------------------------------------------------------------
// Reverse-mode gradient (k_grad.cu)

// One two-qubit update to differentiate (device memory, one per gate of a layer).
struct GradGateDesc {
    const void* a_pre;    // pre-layer site q   (chiL, 2, chiM)
    const void* b_pre;    // pre-layer site q+1 (chiM, 2, chiR)
    const void* u_post;   // post-layer site q  (chiL, 2, k)  = U
    const void* y_post;   // post-layer site q+1 (k, 2, chiR) = c Y
    const void* theta0;   // the gated block T, column-major (2chiL) x (2chiR)
    const void* W;        // the Jacobi columns of the same layer, column-major
    const double* s2;     // sorted squared column norms of W (2chiR)
    const int* perm;      // their columns
    const double* g4;     // the 4x4 gate
    const double* uL;     // the layer's one-qubit gates of q, q+1 (or null)
    const double* uR;
    const void* ub_post;  // adjoint of the post-layer site q
    const void* bb_post;  // adjoint of the post-layer site q+1
    void* ab_pre;         // adjoint of the pre-layer site q (written)
    void* bb_pre;         // adjoint of the pre-layer site q+1 (written)
    double* ubar_l;       // 2x2 adjoints of uL, uR (accumulated)
    double* ubar_r;
    void* scratch;        // 9 cm^2 complex elements
    int chiL, chiM, chiR, k;
    int renorm;
    int cm;               // 2 chi_cap: bound of m = 2 chiL, n = 2 chiR and k
};
// An unpaired site of a layer with a one-qubit gate.
struct Site1Bwd {
    const void* ab_post;  // adjoint of the post-layer site (cl, 2, cr)
    const void* a_pre;    // the pre-layer site
    void* ab_pre;         // adjoint of the pre-layer site (written)
    const double* u;      // the gate
    double* ubar;         // its 2x2 adjoint (accumulated)
    int cl, cr;
};
// The rotations of one layer (device pointers).
struct RotLayer {
    const char* axes;     // n_rot axis letters, the first acts first
    const double* theta;  // [n_qubits][n_rot]
    int n_rot;
    int pad_;
    int64_t u1_off;       // offset (doubles) of this layer's one-qubit gates in the u1 buffer
    int64_t grad_off;     // offset of its angles in the gradient
};
template <typename T>
cudaError_t launch_gate_bwd(const GradGateDesc* d, int n_gates, cudaStream_t s);
template <typename T>
cudaError_t launch_site1_bwd(const Site1Bwd* d, int n_sites, cudaStream_t s);
template <typename T>
cudaError_t launch_env_axpy(void* dst, const void* src, const int* chi, int bond, double coef, int zero_first,
                            int chi_cap, cudaStream_t s);
template <typename T>
cudaError_t launch_site_adj2(const void* E, const double* op, const void* tmp, const int* chi, int q, double coef,
                             void* out, int chi_cap, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_combine(void* ah, const void* an, const void* hsum, const void* nrm, int64_t count,
                               cudaStream_t s);
cudaError_t launch_rot_build(const RotLayer* rl, int n_layers, int n, double* u1, cudaStream_t s);
cudaError_t launch_rot_grad(const RotLayer* rl, int n_layers, int n, const double* ub, double* grad, cudaStream_t s);
// tmp[y, p, a] = sum_b A_q[y, p, b] Rt[b, a]: a site times a (transposed) right environment
template <typename T>
cudaError_t launch_apply_rt(const void* site, const int* chi, int q, const void* rt, void* tmp, int chi_cap,
                            cudaStream_t s);

// Set the thread-local message returned by tnsim_last_error().
void set_last_error(const char* msg);

}  // namespace tnsim

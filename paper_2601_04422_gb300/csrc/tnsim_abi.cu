// Host runtime behind the C ABI (include/tnsim.h).
//
// Memory layout of one state (all device memory is allocated at create time):
//  - site arena: site q owns a fixed slot of cap_q * 2 * cap_{q+1} complex elements,
//    cap_b = min(chi_max, 2^b, 2^(n-b)); the live tensor (chi_q, 2, chi_{q+1}) is
//    stored densely (row-major) at the start of its slot;
//  - chi[0..n]: live bond dimensions, read by the kernels at run time and written by
//    the truncation kernel, so consecutive layers need no host round trip;
//  - one workspace slot per possible gate of a layer (n/2): theta0 and W, each
//    (2 capmax)^2 elements, plus the sorted spectrum / permutation of that gate;
//  - per-bond kept singular values (the spectrum written by the last SVD).
// The host keeps upper bounds ub_b >= chi_b to size grids; the kernels exit early
// outside the live dimensions.  Synchronising calls refresh ub from chi.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>

#include "../../include/tnsim.h"
#include "tnsim_circuit.h"
#include "tnsim_internal.h"

using namespace tnsim;

namespace {

thread_local std::string g_err;

tnsim_status fail(tnsim_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define CUDA_TRY(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(TNSIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

constexpr int kRing = 4;           // pinned staging slots per state

// Process-wide cap on the device memory that states hold (0 = none) and the bytes held.
std::atomic<int64_t> g_dev_cap{0};
std::atomic<int64_t> g_dev_held{0};
constexpr int kMaxChi = 512;       // largest supported chi_max

struct Staging {
    GateDesc* desc = nullptr;      // pinned
    Site1Desc* s1 = nullptr;       // pinned
    double* gates = nullptr;       // pinned: G*32 + n*8 doubles
    cudaEvent_t done = nullptr;    // recorded after the H2D copies that read this slot
    bool used = false;
};

}  // namespace

void tnsim::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

struct tnsim_mps {
    int n = 0;
    tnsim_dtype dt = TNSIM_C64;
    tnsim_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    size_t esz = 8;
    std::vector<int> cap, ub;
    std::vector<size_t> site_off;  // byte offsets into d_sites
    size_t arena_bytes = 0;        // size of d_sites
    int G = 0, capmax = 1;
    size_t ws_elems = 0;
    char* d_sites = nullptr;
    int* d_chi = nullptr;
    char* d_ws = nullptr;          // G slots * (theta0 | W)
    double* d_s2 = nullptr;
    int* d_perm = nullptr;
    double* d_spec = nullptr;      // (n+1) * chi_max
    int* d_spec_k = nullptr;       // (n+1)
    GateOut* d_out = nullptr;      // G
    GateDesc* d_desc = nullptr;    // G
    Site1Desc* d_s1 = nullptr;     // n
    double* d_gates = nullptr;     // G*32 + n*8
    int* d_sticky = nullptr;
    unsigned long long* d_stats = nullptr;   // the counters of tnsim_stats
    JacobiCtl* d_ctl = nullptr;    // control word of the persistent Jacobi launch
    int jac_cfg = 0;               // Jacobi launch configuration (tnsim_set_jacobi_config / tnsim_autotune)
    unsigned jac_spin = 0;         // idle polls of the Jacobi kernel before it gives up (0 = default)
    int tc_spin = 0;               // polls of a tensor-core mbarrier wait before it gives up (0 = default)
    int64_t dev_bytes = 0;         // device bytes held, counted against the process-wide cap
    // tensor-core contraction (complex64 with gemm TF32X3 / BF16X3)
    int tc_mode = -1;              // -1 none, 0 TF32 planes, 1 BF16 planes
    void* d_planes = nullptr;      // [G * 8][tc_rows][tc_k] plane buffer
    CUtensorMap* d_maps = nullptr; // two tensor maps (A boxes, B boxes)
    int tc_rows = 0, tc_k = 0;
    GateOut* h_out = nullptr;      // pinned readback
    int* h_chi = nullptr;          // pinned readback
    Staging ring[kRing];
    int ring_pos = 0;
    // optional per-kernel timing
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int cls; cudaEvent_t a, b; };
    std::vector<Rec> recs;
};

struct tnsim_plan {
    std::vector<tnsim_mps*> states;
    cudaStream_t stream = nullptr;
    int device = 0;
    tnsim_dtype dt = TNSIM_C64;
    int gemm = 0, tc_mode = -1;
    int n_gates = 0, n_s1 = 0;
    int chiL_max = 1, chiM_max = 1, chiR_max = 1, k_max = 1, caplr = 1;
    double tol = 0.0;
    int sweeps = 40;
    GateDesc* d_desc = nullptr;
    GateOut* d_out = nullptr;
    Site1Desc* d_s1 = nullptr;
    JacobiCtl* d_ctl = nullptr;
    bool canon = false;            // some state of the plan is in canonical form
    bool qr = false;               // some state of the plan selected QR preconditioning
    int jac_cfg = 0;               // Jacobi launch configuration of the first state
    unsigned jac_spin = 0;         // idle-poll limit of the first state
    int lead = 0;                  // leading gates of the largest capacity (leading_jobs)
};

struct tnsim_graph {
    cudaStream_t stream = nullptr;
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int cap_of(int n, int b, int chi_max) {
    const int e = std::min(b, n - b);
    if (e >= 30) return chi_max;
    return std::min(chi_max, 1 << e);
}

tnsim_status check_params(const tnsim_params* p) {
    if (p->chi_max < 1 || p->chi_max > kMaxChi)
        return fail(TNSIM_EINVAL, "chi_max must be in [1, 512]");
    if (!(p->cutoff >= 0.0 && p->cutoff < 1.0)) return fail(TNSIM_EINVAL, "cutoff must be in [0, 1)");
    if (p->max_sweeps < 0 || p->max_sweeps > 10000) return fail(TNSIM_EINVAL, "bad max_sweeps");
    if (!(p->jacobi_tol >= 0.0 && p->jacobi_tol < 1.0)) return fail(TNSIM_EINVAL, "bad jacobi_tol");
    if (p->schedule != TNSIM_SCHED_BATCHED && p->schedule != TNSIM_SCHED_PLAIN)
        return fail(TNSIM_EINVAL, "bad schedule");
    if (p->gemm < TNSIM_GEMM_FP32 || p->gemm > TNSIM_GEMM_BF16X3) return fail(TNSIM_EINVAL, "bad gemm mode");
    if (p->form != TNSIM_FORM_PAPER && p->form != TNSIM_FORM_CANONICAL) return fail(TNSIM_EINVAL, "bad form");
    return TNSIM_OK;
}

void free_all(tnsim_mps* m) {
    cudaFree(m->d_sites); cudaFree(m->d_chi); cudaFree(m->d_ws); cudaFree(m->d_s2);
    cudaFree(m->d_perm); cudaFree(m->d_spec); cudaFree(m->d_spec_k); cudaFree(m->d_out);
    cudaFree(m->d_desc); cudaFree(m->d_s1); cudaFree(m->d_gates); cudaFree(m->d_sticky);
    cudaFree(m->d_stats);
    cudaFree(m->d_ctl);
    cudaFree(m->d_planes);
    cudaFree(m->d_maps);
    cudaFreeHost(m->h_out); cudaFreeHost(m->h_chi);
    for (auto& r : m->ring) {
        cudaFreeHost(r.desc); cudaFreeHost(r.s1); cudaFreeHost(r.gates);
        if (r.done) cudaEventDestroy(r.done);
    }
    for (cudaEvent_t e : m->ev_pool) cudaEventDestroy(e);
    for (auto& r : m->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    m->ev_pool.clear();
    m->recs.clear();
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    g_dev_held.fetch_sub(m->dev_bytes);
    m->dev_bytes = 0;
}

cudaEvent_t prof_event(tnsim_mps* m) {
    if (!m->ev_pool.empty()) {
        cudaEvent_t e = m->ev_pool.back();
        m->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Record the start event of a timed launch (no-op when profiling is off).
cudaEvent_t prof_begin(tnsim_mps* m, cudaStream_t st) {
    if (!m->prof_on) return nullptr;
    cudaEvent_t a = prof_event(m);
    if (a) cudaEventRecord(a, st);
    return a;
}

void prof_end(tnsim_mps* m, cudaStream_t st, int cls, cudaEvent_t a) {
    if (!m->prof_on || !a) return;
    cudaEvent_t b = prof_event(m);
    if (!b) return;
    cudaEventRecord(b, st);
    m->recs.push_back({cls, a, b});
}

Staging* acquire_staging(tnsim_mps* m) {
    Staging* s = &m->ring[m->ring_pos];
    m->ring_pos = (m->ring_pos + 1) % kRing;
    if (s->used) cudaEventSynchronize(s->done);
    s->used = true;
    return s;
}

void* site_ptr(tnsim_mps* m, int q) { return m->d_sites + m->site_off[q]; }

// validate a pair list: disjoint adjacent pairs inside the chain
tnsim_status check_pairs(const tnsim_mps* m, int n2, const int32_t* q) {
    if (n2 < 0 || n2 > m->G) return fail(TNSIM_EINVAL, "n2 out of range");
    if (n2 > 0 && !q) return fail(TNSIM_EINVAL, "q is NULL");
    std::vector<char> used(m->n, 0);
    for (int i = 0; i < n2; ++i) {
        if (q[i] < 0 || q[i] >= m->n - 1) return fail(TNSIM_EINVAL, "pair index out of range");
        if (used[q[i]] || used[q[i] + 1]) return fail(TNSIM_EINVAL, "pairs of a layer must be disjoint");
        used[q[i]] = used[q[i] + 1] = 1;
    }
    return TNSIM_OK;
}

bool finite_all(const double* v, size_t count) {
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

double default_tol(const tnsim_mps* m) { return m->p.jacobi_tol; }   // 0 = per-gate default in-kernel
int default_sweeps(const tnsim_mps* m) {
    if (m->p.max_sweeps > 0) return m->p.max_sweeps;
    return m->dt == TNSIM_C64 ? 40 : 60;
}

// One batch of gates (possibly from several states) through K1..K4.
struct GateJob {
    tnsim_mps* m;
    int q;
    int slot;                  // workspace slot of m
    const double* g4;          // device
    const double* uL;          // device or null
    const double* uR;
    double* eps_dev;           // device or null
};

// How many leading jobs of a batch sorted by decreasing size share the first job's size
// (the persistent Jacobi CTAs start spread over them).  cap: compare capacities instead
// of the current bond bounds (the order frozen plans are sorted in).
int leading_jobs(const std::vector<GateJob>& jobs, bool cap) {
    auto key = [cap](const GateJob& j) {
        const int* b = cap ? j.m->cap.data() : j.m->ub.data();
        return (double)b[j.q] * b[j.q + 2] * b[j.q + 2];
    };
    int k = 0;
    while (k < (int)jobs.size() && key(jobs[k]) == key(jobs[0])) ++k;
    return k;
}

// Fill and upload the descriptors of a batch of gates (possibly from several states).
// qr_force >= 0 replaces every state's QR-preconditioning choice (the autotuner's descriptors).
tnsim_status upload_desc(cudaStream_t st, const std::vector<GateJob>& jobs, GateDesc* h_desc,
                         GateDesc* d_desc, GateOut* d_out_base, int qr_force = -1) {
    const int ng = (int)jobs.size();
    if (ng == 0) return TNSIM_OK;
    for (int i = 0; i < ng; ++i) {
        const GateJob& j = jobs[i];
        tnsim_mps* m = j.m;
        const size_t es = m->esz;
        char* ws = m->d_ws + (size_t)j.slot * 2 * m->ws_elems * es;
        GateDesc& d = h_desc[i];
        std::memset(&d, 0, sizeof(d));
        d.siteA = site_ptr(m, j.q);
        d.siteB = site_ptr(m, j.q + 1);
        d.chi = m->d_chi;
        d.g4 = j.g4;
        d.uL = j.uL;
        d.uR = j.uR;
        d.theta0 = ws;
        d.W = ws + m->ws_elems * es;
        d.s2 = m->d_s2 + (size_t)j.slot * 2 * m->capmax;
        d.perm = m->d_perm + (size_t)j.slot * 2 * m->capmax;
        d.spectrum = m->d_spec + (size_t)(j.q + 1) * m->p.chi_max;
        d.spec_k = m->d_spec_k + (j.q + 1);
        d.eps_out = j.eps_dev;
        d.out = d_out_base ? (d_out_base + i) : (m->d_out + j.slot);
        d.sticky = m->d_sticky;
        d.stats = m->d_stats;
        d.cutoff = m->p.cutoff;
        d.q = j.q;
        d.chi_max = m->p.chi_max;
        d.renorm = m->p.renormalize ? 1 : 0;
        d.tc_planes = m->d_planes;
        d.tc_map_a = m->d_maps;
        d.tc_map_b = m->d_maps ? m->d_maps + 1 : nullptr;
        d.tc_slot = j.slot;
        d.tc_rows = m->tc_rows;
        d.tc_k = m->tc_k;
        d.canon = m->p.form == TNSIM_FORM_CANONICAL ? 1 : 0;
        d.lam = m->d_spec + (size_t)j.q * m->p.chi_max;
        d.lam_k = m->d_spec_k + j.q;
        d.qr = qr_force >= 0 ? qr_force : (m->jac_cfg >> 1) & 1;
        d.wait_polls = m->tc_spin;
    }
    CUDA_TRY(cudaMemcpyAsync(d_desc, h_desc, sizeof(GateDesc) * ng, cudaMemcpyHostToDevice, st));
    return TNSIM_OK;
}

template <typename T>
tnsim_status launch_gates(cudaStream_t st, const std::vector<GateJob>& jobs, const GateDesc* d_desc,
                          double tol, int sweeps) {
    const int ng = (int)jobs.size();
    if (ng == 0) return TNSIM_OK;
    int chiL_max = 1, chiM_max = 1, chiR_max = 1, k_max = 1;
    for (const GateJob& j : jobs) {
        chiL_max = std::max(chiL_max, j.m->ub[j.q]);
        chiM_max = std::max(chiM_max, j.m->ub[j.q + 1]);
        chiR_max = std::max(chiR_max, j.m->ub[j.q + 2]);
        k_max = std::max(k_max, std::min({j.m->cap[j.q + 1], 2 * j.m->ub[j.q], 2 * j.m->ub[j.q + 2]}));
    }
    const int m_max = 2 * chiL_max, n_max = 2 * chiR_max;
    tnsim_mps* pm = jobs[0].m;   // the state whose profiler records this batch
    cudaEvent_t ev = prof_begin(pm, st);
    if (sizeof(T) == 8 || pm->p.gemm == TNSIM_GEMM_FP32) {
        CUDA_TRY(launch_theta<T>(d_desc, ng, chiL_max, chiR_max, st));
    } else if (pm->p.gemm == TNSIM_GEMM_FP32_3M) {
        CUDA_TRY(launch_theta_3m(d_desc, ng, chiL_max, chiR_max, st));
    } else {
        CUDA_TRY(launch_theta_tc(pm->tc_mode, d_desc, ng, chiL_max, chiM_max, chiR_max, st));
    }
    prof_end(pm, st, TNSIM_K_THETA, ev);
    bool canon = false, qr = false;
    for (const GateJob& j : jobs) {
        canon = canon || j.m->p.form == TNSIM_FORM_CANONICAL;
        qr = qr || (j.m->jac_cfg & 2) != 0;
    }
    if (canon) CUDA_TRY(launch_scale_rows<T>(d_desc, ng, st));
    CUDA_TRY(cudaMemsetAsync(pm->d_ctl, 0, sizeof(JacobiCtl), st));
    if (qr) {
        ev = prof_begin(pm, st);
        CUDA_TRY(launch_qr<T>(d_desc, ng, m_max, st));
        prof_end(pm, st, TNSIM_K_QR, ev);
    }
    ev = prof_begin(pm, st);
    CUDA_TRY(launch_jacobi<T>(d_desc, ng, m_max, n_max, tol, sweeps, pm->d_ctl, st, pm->jac_cfg,
                              leading_jobs(jobs, false), pm->jac_spin));
    prof_end(pm, st, TNSIM_K_JACOBI, ev);
    ev = prof_begin(pm, st);
    CUDA_TRY(launch_truncate<T>(d_desc, ng, n_max, st));
    prof_end(pm, st, TNSIM_K_TRUNCATE, ev);
    ev = prof_begin(pm, st);
    CUDA_TRY(launch_left<T>(d_desc, ng, m_max, k_max, st));
    prof_end(pm, st, TNSIM_K_LEFT, ev);
    ev = prof_begin(pm, st);
    CUDA_TRY(launch_right<T>(d_desc, ng, k_max, n_max, st));
    if (canon) CUDA_TRY(launch_left_canon<T>(d_desc, ng, m_max, k_max, st));
    if (qr)
        CUDA_TRY(launch_sites_pre<T>(d_desc, ng, m_max, k_max, n_max, st,
                                     pm->p.gemm == TNSIM_GEMM_TF32X3 || pm->p.gemm == TNSIM_GEMM_BF16X3));
    prof_end(pm, st, TNSIM_K_RIGHT, ev);
    // bounds for the next layer
    for (const GateJob& j : jobs) {
        tnsim_mps* m = j.m;
        m->ub[j.q + 1] = std::min({m->cap[j.q + 1], 2 * m->ub[j.q], 2 * m->ub[j.q + 2]});
    }
    return TNSIM_OK;
}

tnsim_status launch_gates_dt(tnsim_dtype dt, cudaStream_t st, const std::vector<GateJob>& jobs,
                             const GateDesc* d_desc, double tol, int sweeps) {
    return dt == TNSIM_C64 ? launch_gates<float>(st, jobs, d_desc, tol, sweeps)
                           : launch_gates<double>(st, jobs, d_desc, tol, sweeps);
}

// the one-qubit updates of the qubits outside every pair
tnsim_status launch_unpaired(tnsim_mps* m, Staging* stg, int n2, const int32_t* q, const double* u1_dev) {
    std::vector<char> used(m->n, 0);
    for (int i = 0; i < n2; ++i) used[q[i]] = used[q[i] + 1] = 1;
    int ns = 0, caplr = 1;
    for (int s = 0; s < m->n; ++s) {
        if (used[s]) continue;
        Site1Desc& d = stg->s1[ns++];
        d.site = site_ptr(m, s);
        d.chi = m->d_chi;
        d.u = u1_dev + (size_t)s * 8;
        d.q = s;
        d.pad_ = 0;
        caplr = std::max(caplr, m->ub[s] * m->ub[s + 1]);
    }
    if (ns == 0) return TNSIM_OK;
    CUDA_TRY(cudaMemcpyAsync(m->d_s1, stg->s1, sizeof(Site1Desc) * ns, cudaMemcpyHostToDevice, m->stream));
    cudaEvent_t ev = prof_begin(m, m->stream);
    if (m->dt == TNSIM_C64) CUDA_TRY(launch_site1q<float>(m->d_s1, ns, caplr, m->stream));
    else CUDA_TRY(launch_site1q<double>(m->d_s1, ns, caplr, m->stream));
    prof_end(m, m->stream, TNSIM_K_SITE1Q, ev);
    return TNSIM_OK;
}

// The gates of one layer of m as jobs (slot i for pair i), largest first: the
// persistent Jacobi kernel serves gates in descriptor order.
std::vector<GateJob> layer_jobs(tnsim_mps* m, int n2, const int32_t* q, const double* g4_dev,
                                const double* u1_dev, double* eps_dev) {
    std::vector<GateJob> jobs(n2);
    for (int i = 0; i < n2; ++i) {
        jobs[i].m = m;
        jobs[i].q = q[i];
        jobs[i].slot = i;
        jobs[i].g4 = g4_dev + (size_t)i * 32;
        jobs[i].uL = u1_dev ? u1_dev + (size_t)q[i] * 8 : nullptr;
        jobs[i].uR = u1_dev ? u1_dev + (size_t)(q[i] + 1) * 8 : nullptr;
        jobs[i].eps_dev = eps_dev ? eps_dev + i : nullptr;
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const GateJob& a, const GateJob& b) {
        const double ca = (double)a.m->ub[a.q] * a.m->ub[a.q + 2] * a.m->ub[a.q + 2];
        const double cb = (double)b.m->ub[b.q] * b.m->ub[b.q + 2] * b.m->ub[b.q + 2];
        return ca > cb;
    });
    return jobs;
}

// Enqueue one layer whose gate data is in device memory.
tnsim_status enqueue_layer(tnsim_mps* m, Staging* stg, int n2, const int32_t* q, const double* g4_dev,
                           const double* u1_dev, double* eps_dev) {
    cudaStream_t st = m->stream;
    if (u1_dev) {
        tnsim_status s = launch_unpaired(m, stg, n2, q, u1_dev);
        if (s != TNSIM_OK) return s;
    }
    if (n2 == 0) return TNSIM_OK;
    std::vector<GateJob> jobs = layer_jobs(m, n2, q, g4_dev, u1_dev, eps_dev);
    CUDA_TRY(cudaMemsetAsync(m->d_out, 0, sizeof(GateOut) * n2, st));
    const double tol = default_tol(m);
    const int sweeps = default_sweeps(m);
    tnsim_status s;
    s = upload_desc(st, jobs, stg->desc, m->d_desc, nullptr);
    if (s != TNSIM_OK) return s;
    if (m->p.schedule == TNSIM_SCHED_PLAIN) {
        // one pair at a time: each pair is its own launch sequence
        for (int i = 0; i < n2; ++i) {
            std::vector<GateJob> one(1, jobs[i]);
            s = launch_gates_dt(m->dt, st, one, m->d_desc + i, tol, sweeps);
            if (s != TNSIM_OK) return s;
        }
    } else {
        s = launch_gates_dt(m->dt, st, jobs, m->d_desc, tol, sweeps);
        if (s != TNSIM_OK) return s;
    }
    return TNSIM_OK;
}

tnsim_status refresh_dims(tnsim_mps* m) {
    CUDA_TRY(cudaMemcpyAsync(m->h_chi, m->d_chi, sizeof(int) * (m->n + 1), cudaMemcpyDeviceToHost, m->stream));
    CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (int b = 0; b <= m->n; ++b) m->ub[b] = m->h_chi[b];
    return TNSIM_OK;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DevGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

}  // namespace

// ===========================================================================
extern "C" {

const char* tnsim_last_error(void) { return g_err.c_str(); }
const char* tnsim_version(void) { return "tnsim-gb300 0.1 (sm_103a)"; }

tnsim_status tnsim_params_default(tnsim_dtype dt, tnsim_params* out) {
    if (!out) return fail(TNSIM_EINVAL, "out is NULL");
    if (dt != TNSIM_C64 && dt != TNSIM_C128) return fail(TNSIM_EINVAL, "unknown dtype");
    out->chi_max = 64;
    out->cutoff = 0.0;
    out->renormalize = 1;
    out->max_sweeps = 0;
    out->jacobi_tol = 0.0;
    out->schedule = TNSIM_SCHED_BATCHED;
    out->gemm = TNSIM_GEMM_FP32;
    out->form = TNSIM_FORM_PAPER;
    return TNSIM_OK;
}

tnsim_status tnsim_mps_create(int32_t n_qubits, tnsim_dtype dt, const tnsim_params* p,
                              void* cuda_stream, tnsim_mps** out) {
    g_err.clear();
    if (!out) return fail(TNSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_qubits < 2 || n_qubits > (1 << 20)) return fail(TNSIM_EINVAL, "n_qubits must be >= 2");
    if (dt != TNSIM_C64 && dt != TNSIM_C128) return fail(TNSIM_EINVAL, "unknown dtype");
    tnsim_params prm;
    tnsim_params_default(dt, &prm);
    if (p) prm = *p;
    tnsim_status s = check_params(&prm);
    if (s != TNSIM_OK) return s;

    tnsim_mps* m = new (std::nothrow) tnsim_mps();
    if (!m) return fail(TNSIM_ENOMEM, "host allocation failed");
    m->n = n_qubits;
    m->dt = dt;
    m->p = prm;
    m->esz = dt == TNSIM_C64 ? 8 : 16;
    cudaGetDevice(&m->device);
    m->cap.resize(n_qubits + 1);
    m->ub.assign(n_qubits + 1, 1);
    for (int b = 0; b <= n_qubits; ++b) {
        m->cap[b] = cap_of(n_qubits, b, prm.chi_max);
        m->capmax = std::max(m->capmax, m->cap[b]);
    }
    m->site_off.resize(n_qubits);
    size_t off = 0;
    for (int q = 0; q < n_qubits; ++q) {
        m->site_off[q] = off;
        size_t bytes = (size_t)m->cap[q] * 2 * m->cap[q + 1] * m->esz;
        off += (bytes + 255) / 256 * 256;
    }
    m->G = n_qubits / 2;
    m->ws_elems = (size_t)(2 * m->capmax) * (2 * m->capmax);
    const size_t nG = (size_t)m->G;
    const size_t gate_doubles = nG * 32 + (size_t)n_qubits * 8;

#define ALLOC(ptr, bytes)                                                        \
    do {                                                                         \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                    \
        if (e_ != cudaSuccess) {                                                 \
            free_all(m); delete m;                                               \
            return fail(TNSIM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e_)); \
        }                                                                        \
    } while (0)
#define HALLOC(ptr, bytes)                                                       \
    do {                                                                         \
        cudaError_t e_ = cudaMallocHost((void**)&(ptr), (bytes));                \
        if (e_ != cudaSuccess) {                                                 \
            free_all(m); delete m;                                               \
            return fail(TNSIM_ENOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e_)); \
        }                                                                        \
    } while (0)

    m->arena_bytes = off;
    // every device allocation of the state, checked against the process-wide cap first
    const bool use_tc = dt == TNSIM_C64 && (prm.gemm == TNSIM_GEMM_TF32X3 || prm.gemm == TNSIM_GEMM_BF16X3);
    {
        const size_t capmax2 = (size_t)(2 * m->capmax);
        int64_t need = (int64_t)(off + sizeof(int) * (n_qubits + 1) + nG * 2 * m->ws_elems * m->esz +
                                 nG * capmax2 * (sizeof(double) + sizeof(int)) +
                                 (size_t)(n_qubits + 1) * prm.chi_max * sizeof(double) + sizeof(int) * (n_qubits + 1) +
                                 nG * (sizeof(GateOut) + sizeof(GateDesc)) + (size_t)n_qubits * sizeof(Site1Desc) +
                                 gate_doubles * sizeof(double) + sizeof(int) + sizeof(tnsim_stats) + sizeof(JacobiCtl));
        if (use_tc) need += (int64_t)(nG * 8 * capmax2 * ((m->capmax + 63) / 64 * 64) * sizeof(float) +
                                      2 * sizeof(CUtensorMap));
        const int64_t cap = g_dev_cap.load();
        const int64_t held = g_dev_held.fetch_add(need) + need;
        if (cap > 0 && held > cap) {
            g_dev_held.fetch_sub(need);
            delete m;
            return fail(TNSIM_ENOMEM, "the state needs " + std::to_string(need) + " device bytes; with " +
                                          std::to_string(held - need) + " held, that exceeds the cap of " +
                                          std::to_string(cap) + " bytes (tnsim_set_device_memory_cap)");
        }
        m->dev_bytes = need;
    }
    ALLOC(m->d_sites, off);
    ALLOC(m->d_chi, sizeof(int) * (n_qubits + 1));
    ALLOC(m->d_ws, nG * 2 * m->ws_elems * m->esz);
    ALLOC(m->d_s2, nG * 2 * m->capmax * sizeof(double));
    ALLOC(m->d_perm, nG * 2 * m->capmax * sizeof(int));
    ALLOC(m->d_spec, (size_t)(n_qubits + 1) * prm.chi_max * sizeof(double));
    ALLOC(m->d_spec_k, sizeof(int) * (n_qubits + 1));
    ALLOC(m->d_out, nG * sizeof(GateOut));
    ALLOC(m->d_desc, nG * sizeof(GateDesc));
    ALLOC(m->d_s1, (size_t)n_qubits * sizeof(Site1Desc));
    ALLOC(m->d_gates, gate_doubles * sizeof(double));
    ALLOC(m->d_sticky, sizeof(int));
    ALLOC(m->d_stats, sizeof(tnsim_stats));
    ALLOC(m->d_ctl, sizeof(JacobiCtl));
    HALLOC(m->h_out, nG * sizeof(GateOut));
    HALLOC(m->h_chi, sizeof(int) * (n_qubits + 1));
    for (auto& r : m->ring) {
        HALLOC(r.desc, nG * sizeof(GateDesc));
        HALLOC(r.s1, (size_t)n_qubits * sizeof(Site1Desc));
        HALLOC(r.gates, gate_doubles * sizeof(double));
        if (cudaEventCreateWithFlags(&r.done, cudaEventDisableTiming) != cudaSuccess) {
            free_all(m); delete m;
            return fail(TNSIM_ECUDA, "cudaEventCreate failed");
        }
    }
    if (use_tc) {
        m->tc_mode = prm.gemm == TNSIM_GEMM_TF32X3 ? 0 : 1;
        m->tc_rows = 2 * m->capmax;
        m->tc_k = (m->capmax + 63) / 64 * 64;
        const size_t pbytes = nG * 8 * (size_t)m->tc_rows * m->tc_k * sizeof(float);
        ALLOC(m->d_planes, pbytes);
        ALLOC(m->d_maps, 2 * sizeof(CUtensorMap));
        CUtensorMap hm[2];
        cudaError_t e1 = cudaMemset(m->d_planes, 0, pbytes);
        if (e1 == cudaSuccess)
            e1 = encode_plane_maps(m->tc_mode, m->d_planes, (int)nG, m->tc_rows, m->tc_k, &hm[0], &hm[1]);
        if (e1 == cudaSuccess) e1 = cudaMemcpy(m->d_maps, hm, sizeof(hm), cudaMemcpyHostToDevice);
        if (e1 != cudaSuccess) {
            free_all(m); delete m;
            return fail(TNSIM_ECUDA, std::string("tensor-core operand set-up: ") + cudaGetErrorString(e1));
        }
    }
#undef ALLOC
#undef HALLOC
    if (cuda_stream) {
        m->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            free_all(m); delete m;
            return fail(TNSIM_ECUDA, "cudaStreamCreate failed");
        }
        m->own_stream = true;
    }
    // |0...0>: every site (1,2,1) = (1, 0)
    std::vector<char> h0(m->esz * 2, 0);
    if (dt == TNSIM_C64) { float one = 1.0f; std::memcpy(h0.data(), &one, 4); }
    else { double one = 1.0; std::memcpy(h0.data(), &one, 8); }
    std::vector<int> ones(n_qubits + 1, 1);
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < n_qubits && e == cudaSuccess; ++q)
        e = cudaMemcpy(m->d_sites + m->site_off[q], h0.data(), h0.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_chi, ones.data(), sizeof(int) * (n_qubits + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_spec_k, 0, sizeof(int) * (n_qubits + 1));
    if (e == cudaSuccess) e = cudaMemset(m->d_sticky, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(m->d_stats, 0, sizeof(tnsim_stats));
    if (e == cudaSuccess) e = cudaMemset(m->d_out, 0, nG * sizeof(GateOut));
    // finite contents from the start: a contraction that timed out leaves its W unwritten
    if (e == cudaSuccess) e = cudaMemset(m->d_ws, 0, nG * 2 * m->ws_elems * m->esz);
    if (e != cudaSuccess) {
        free_all(m); delete m;
        return fail(TNSIM_ECUDA, std::string("initialisation: ") + cudaGetErrorString(e));
    }
    *out = m;
    return TNSIM_OK;
}

tnsim_status tnsim_mps_destroy(tnsim_mps* m) {
    if (!m) return TNSIM_OK;
    DevGuard g(m->device);
    cudaStreamSynchronize(m->stream);
    free_all(m);
    delete m;
    return TNSIM_OK;
}

tnsim_status tnsim_apply_layer_device(tnsim_mps* m, int32_t n2, const int32_t* q,
                                      const double* g4x4_dev, const double* u1_dev, double* eps_dev) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    DevGuard g(m->device);
    tnsim_status s = check_pairs(m, n2, q);
    if (s != TNSIM_OK) return s;
    if (n2 > 0 && !g4x4_dev) return fail(TNSIM_EINVAL, "g4x4_dev is NULL");
    Staging* stg = acquire_staging(m);
    s = enqueue_layer(m, stg, n2, q, g4x4_dev, u1_dev, eps_dev);
    CUDA_TRY(cudaEventRecord(stg->done, m->stream));
    return s;
}

tnsim_status tnsim_apply_layer(tnsim_mps* m, int32_t n2, const int32_t* q, const double* g4x4,
                               const double* u1, double* eps_out) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    DevGuard g(m->device);
    tnsim_status s = check_pairs(m, n2, q);
    if (s != TNSIM_OK) return s;
    if (n2 > 0 && !g4x4) return fail(TNSIM_EINVAL, "g4x4 is NULL");
    if (n2 > 0 && !finite_all(g4x4, (size_t)n2 * 32)) return fail(TNSIM_EINVAL, "non-finite gate entry");
    if (u1 && !finite_all(u1, (size_t)m->n * 8)) return fail(TNSIM_EINVAL, "non-finite one-qubit gate entry");
    Staging* stg = acquire_staging(m);
    double* dg = m->d_gates;
    double* du = m->d_gates + (size_t)m->G * 32;
    if (n2 > 0) std::memcpy(stg->gates, g4x4, sizeof(double) * 32 * n2);
    if (u1) std::memcpy(stg->gates + (size_t)m->G * 32, u1, sizeof(double) * 8 * m->n);
    if (n2 > 0) CUDA_TRY(cudaMemcpyAsync(dg, stg->gates, sizeof(double) * 32 * n2, cudaMemcpyHostToDevice, m->stream));
    if (u1) CUDA_TRY(cudaMemcpyAsync(du, stg->gates + (size_t)m->G * 32, sizeof(double) * 8 * m->n,
                                     cudaMemcpyHostToDevice, m->stream));
    s = enqueue_layer(m, stg, n2, q, dg, u1 ? du : nullptr, nullptr);
    CUDA_TRY(cudaEventRecord(stg->done, m->stream));
    if (s != TNSIM_OK) return s;
    if (n2 > 0) CUDA_TRY(cudaMemcpyAsync(m->h_out, m->d_out, sizeof(GateOut) * n2, cudaMemcpyDeviceToHost, m->stream));
    s = refresh_dims(m);   // synchronises
    if (s != TNSIM_OK) return s;
    int worst = 0;
    for (int i = 0; i < n2; ++i) {
        if (eps_out) eps_out[i] = m->h_out[i].eps;
        worst = std::max(worst, m->h_out[i].status);
    }
    if (worst) CUDA_TRY(cudaMemset(m->d_sticky, 0, sizeof(int)));
    if (worst == 5) return fail(TNSIM_ETIMEOUT, "a bounded device wait ran out: an idle Jacobi CTA saw no progress or a tensor-core wait expired (layer incomplete)");
    if (worst == 4) return fail(TNSIM_ENOCONV, "a Jacobi SVD reached max_sweeps (layer applied)");
    return TNSIM_OK;
}

tnsim_status tnsim_apply_circuit(tnsim_mps* m, int32_t n_ops, const int32_t* qa, const int32_t* qb,
                                 const double* mats, int32_t* n_layers_out, int32_t* n_gates_out,
                                 double* eps_sum_out) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    DevGuard g(m->device);
    tnsim::CircuitLayers cl;
    std::string err;
    tnsim_status s = tnsim::layerize_circuit(m->n, n_ops, qa, qb, mats, cl, err);
    if (s != TNSIM_OK) return fail(s, err);
    const int nl = (int)cl.n2.size(), ng = (int)cl.q.size();
    if (n_layers_out) *n_layers_out = nl;
    if (n_gates_out) *n_gates_out = ng;
    if (eps_sum_out) *eps_sum_out = 0.0;
    if (nl == 0) return TNSIM_OK;
    for (int L = 0; L < nl; ++L) {
        s = check_pairs(m, cl.n2[L], cl.q.data() + cl.q_off[L]);
        if (s != TNSIM_OK) return s;
    }
    // every gate of the list on the device at once: the 4x4s, the one-qubit layers in
    // use and one discarded weight per local two-qubit gate
    int nu = 0;
    for (char h : cl.has_u1) nu += h ? 1 : 0;
    const size_t n8 = (size_t)m->n * 8;
    std::vector<double> hbuf((size_t)ng * 32 + (size_t)nu * n8);
    std::memcpy(hbuf.data(), cl.g4.data(), sizeof(double) * cl.g4.size());
    for (int L = 0, ui = 0; L < nl; ++L)
        if (cl.has_u1[L]) std::memcpy(hbuf.data() + (size_t)ng * 32 + (size_t)(ui++) * n8, cl.u1.data() + L * n8,
                                      sizeof(double) * n8);
    double* dbuf = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&dbuf, sizeof(double) * (hbuf.size() + ng), m->stream));
    double* d_g4 = dbuf;
    double* d_u1 = dbuf + (size_t)ng * 32;
    double* d_eps = d_u1 + (size_t)nu * n8;
    // from pageable memory: returns once hbuf has been consumed
    CUDA_TRY(cudaMemcpyAsync(dbuf, hbuf.data(), sizeof(double) * hbuf.size(), cudaMemcpyHostToDevice, m->stream));
    CUDA_TRY(cudaMemsetAsync(d_eps, 0, sizeof(double) * ng, m->stream));
    for (int L = 0, ui = 0; L < nl; ++L) {
        Staging* stg = acquire_staging(m);
        const double* u1 = cl.has_u1[L] ? d_u1 + (size_t)(ui++) * n8 : nullptr;
        s = enqueue_layer(m, stg, cl.n2[L], cl.q.data() + cl.q_off[L], d_g4 + (size_t)cl.q_off[L] * 32, u1,
                          d_eps + cl.q_off[L]);
        CUDA_TRY(cudaEventRecord(stg->done, m->stream));
        if (s != TNSIM_OK) {
            cudaFreeAsync(dbuf, m->stream);
            return s;
        }
    }
    std::vector<double> eps((size_t)ng);
    int sticky = 0;
    CUDA_TRY(cudaMemcpyAsync(eps.data(), d_eps, sizeof(double) * ng, cudaMemcpyDeviceToHost, m->stream));
    CUDA_TRY(cudaMemcpyAsync(&sticky, m->d_sticky, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CUDA_TRY(cudaFreeAsync(dbuf, m->stream));
    s = refresh_dims(m);   // synchronises
    if (s != TNSIM_OK) return s;
    double tot = 0.0;
    for (double e : eps) tot += e;
    if (eps_sum_out) *eps_sum_out = tot;
    if (sticky) CUDA_TRY(cudaMemset(m->d_sticky, 0, sizeof(int)));
    if (sticky == 5) return fail(TNSIM_ETIMEOUT, "a bounded device wait ran out: an idle Jacobi CTA saw no progress or a tensor-core wait expired (circuit incomplete)");
    if (sticky == 4) return fail(TNSIM_ENOCONV, "a Jacobi SVD reached max_sweeps (circuit applied)");
    return TNSIM_OK;
}

tnsim_status tnsim_apply_layers_batched(tnsim_mps* const* ms, int32_t n_circ, int32_t n_steps,
                                        const int32_t* n2, const int32_t* const* q_ptrs,
                                        const double* const* g_ptrs, const double* const* u1_ptrs) {
    if (n_circ < 0 || n_steps < 0) return fail(TNSIM_EINVAL, "negative count");
    if (n_circ == 0 || n_steps == 0) return TNSIM_OK;
    if (!ms || !n2 || !q_ptrs || !g_ptrs || !u1_ptrs) return fail(TNSIM_EINVAL, "NULL argument");
    for (int i = 0; i < n_circ; ++i) {
        if (!ms[i]) return fail(TNSIM_EINVAL, "state is NULL");
        if (ms[i]->dt != ms[0]->dt) return fail(TNSIM_EINVAL, "all states must share the dtype");
        if (ms[i]->device != ms[0]->device) return fail(TNSIM_EINVAL, "all states must be on one device");
        if (ms[i]->p.gemm != ms[0]->p.gemm) return fail(TNSIM_EINVAL, "all states must share the gemm mode");
        for (int j = 0; j < i; ++j)
            if (ms[j] == ms[i]) return fail(TNSIM_EINVAL, "a state appears twice");
    }
    // validate everything before launching anything
    size_t max_gates = 0, max_u1 = 0, max_sites = 0;
    for (int t = 0; t < n_steps; ++t) {
        size_t ng = 0, nu = 0, ns = 0;
        for (int i = 0; i < n_circ; ++i) {
            const int k = t * n_circ + i;
            tnsim_status s = check_pairs(ms[i], n2[k], q_ptrs[k]);
            if (s != TNSIM_OK) return s;
            if (n2[k] > 0 && !g_ptrs[k]) return fail(TNSIM_EINVAL, "gate pointer is NULL");
            if (n2[k] > 0 && !finite_all(g_ptrs[k], (size_t)n2[k] * 32)) return fail(TNSIM_EINVAL, "non-finite gate entry");
            if (u1_ptrs[k] && !finite_all(u1_ptrs[k], (size_t)ms[i]->n * 8))
                return fail(TNSIM_EINVAL, "non-finite one-qubit gate entry");
            ng += n2[k];
            if (u1_ptrs[k]) { nu += ms[i]->n; ns += ms[i]->n; }
        }
        max_gates = std::max(max_gates, ng);
        max_u1 = std::max(max_u1, nu);
        max_sites = std::max(max_sites, ns);
    }
    tnsim_mps* m0 = ms[0];
    DevGuard g(m0->device);
    for (int i = 0; i < n_circ; ++i)
        if (ms[i]->stream != m0->stream) CUDA_TRY(cudaStreamSynchronize(ms[i]->stream));
    cudaStream_t st = m0->stream;

    // per-call device buffers (stream-ordered allocator) and pinned staging
    const size_t gate_doubles = max_gates * 32 + max_u1 * 8 + 1;
    double* d_g = nullptr;
    GateDesc* d_desc = nullptr;
    GateOut* d_out = nullptr;
    Site1Desc* d_s1 = nullptr;
    double* h_g = nullptr;
    GateDesc* h_desc = nullptr;
    Site1Desc* h_s1 = nullptr;
    GateOut* h_out = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        cudaFreeAsync(d_g, st); cudaFreeAsync(d_desc, st); cudaFreeAsync(d_out, st); cudaFreeAsync(d_s1, st);
        cudaStreamSynchronize(st);
        cudaFreeHost(h_g); cudaFreeHost(h_desc); cudaFreeHost(h_s1); cudaFreeHost(h_out);
    };
    cudaError_t e = cudaMallocAsync((void**)&d_g, sizeof(double) * gate_doubles, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_desc, sizeof(GateDesc) * (max_gates + 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_out, sizeof(GateOut) * (max_gates + 1), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&d_s1, sizeof(Site1Desc) * (max_sites + 1), st);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h_g, sizeof(double) * gate_doubles);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h_desc, sizeof(GateDesc) * (max_gates + 1));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h_s1, sizeof(Site1Desc) * (max_sites + 1));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h_out, sizeof(GateOut) * (max_gates + 1));
    if (e != cudaSuccess) {
        cleanup();
        return fail(TNSIM_ENOMEM, std::string("batched buffers: ") + cudaGetErrorString(e));
    }
    const double tol = m0->p.jacobi_tol;
    int sweeps = 0;
    for (int i = 0; i < n_circ; ++i) sweeps = std::max(sweeps, default_sweeps(ms[i]));
    int worst = 0;
    tnsim_status ret = TNSIM_OK;
    for (int t = 0; t < n_steps && ret == TNSIM_OK; ++t) {
        // stage this step's gates and one-qubit gates
        size_t gpos = 0, upos = max_gates * 32;
        std::vector<GateJob> jobs;
        int ns = 0, caplr = 1;
        for (int i = 0; i < n_circ; ++i) {
            const int k = t * n_circ + i;
            tnsim_mps* m = ms[i];
            const double* u_dev = nullptr;
            if (u1_ptrs[k]) {
                std::memcpy(h_g + upos, u1_ptrs[k], sizeof(double) * 8 * m->n);
                u_dev = d_g + upos;
                upos += (size_t)m->n * 8;
                std::vector<char> used(m->n, 0);
                for (int j = 0; j < n2[k]; ++j) used[q_ptrs[k][j]] = used[q_ptrs[k][j] + 1] = 1;
                for (int sidx = 0; sidx < m->n; ++sidx) {
                    if (used[sidx]) continue;
                    Site1Desc& d = h_s1[ns++];
                    d.site = site_ptr(m, sidx);
                    d.chi = m->d_chi;
                    d.u = u_dev + (size_t)sidx * 8;
                    d.q = sidx;
                    d.pad_ = 0;
                    caplr = std::max(caplr, m->ub[sidx] * m->ub[sidx + 1]);
                }
            }
            if (n2[k] > 0) std::memcpy(h_g + gpos, g_ptrs[k], sizeof(double) * 32 * n2[k]);
            for (int j = 0; j < n2[k]; ++j) {
                GateJob jb;
                jb.m = m;
                jb.q = q_ptrs[k][j];
                jb.slot = j;
                jb.g4 = d_g + gpos + (size_t)j * 32;
                jb.uL = u_dev ? u_dev + (size_t)jb.q * 8 : nullptr;
                jb.uR = u_dev ? u_dev + (size_t)(jb.q + 1) * 8 : nullptr;
                jb.eps_dev = nullptr;
                jobs.push_back(jb);
            }
            gpos += (size_t)n2[k] * 32;
        }
        e = cudaMemcpyAsync(d_g, h_g, sizeof(double) * gate_doubles, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && ns > 0) e = cudaMemcpyAsync(d_s1, h_s1, sizeof(Site1Desc) * ns, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { ret = fail(TNSIM_ECUDA, cudaGetErrorString(e)); break; }
        if (ns > 0) {
            cudaEvent_t ev = prof_begin(m0, st);
            e = (m0->dt == TNSIM_C64) ? launch_site1q<float>(d_s1, ns, caplr, st) : launch_site1q<double>(d_s1, ns, caplr, st);
            prof_end(m0, st, TNSIM_K_SITE1Q, ev);
            if (e != cudaSuccess) { ret = fail(TNSIM_ECUDA, cudaGetErrorString(e)); break; }
        }
        if (!jobs.empty()) {
            std::stable_sort(jobs.begin(), jobs.end(), [](const GateJob& a, const GateJob& b) {
                const double ca = (double)a.m->ub[a.q] * a.m->ub[a.q + 2] * a.m->ub[a.q + 2];
                const double cb = (double)b.m->ub[b.q] * b.m->ub[b.q + 2] * b.m->ub[b.q + 2];
                return ca > cb;
            });
            e = cudaMemsetAsync(d_out, 0, sizeof(GateOut) * jobs.size(), st);
            if (e != cudaSuccess) { ret = fail(TNSIM_ECUDA, cudaGetErrorString(e)); break; }
            ret = upload_desc(st, jobs, h_desc, d_desc, d_out);
            if (ret != TNSIM_OK) break;
            ret = launch_gates_dt(m0->dt, st, jobs, d_desc, tol, sweeps);
            if (ret != TNSIM_OK) break;
            // the pinned staging is reused by the next step
            e = cudaMemcpyAsync(h_out, d_out, sizeof(GateOut) * jobs.size(), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { ret = fail(TNSIM_ECUDA, cudaGetErrorString(e)); break; }
            for (size_t j = 0; j < jobs.size(); ++j) worst = std::max(worst, h_out[j].status);
        } else {
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { ret = fail(TNSIM_ECUDA, cudaGetErrorString(e)); break; }
        }
    }
    cleanup();
    if (ret != TNSIM_OK) return ret;
    for (int i = 0; i < n_circ; ++i) {
        tnsim_status s = refresh_dims(ms[i]);
        if (s != TNSIM_OK) return s;
        CUDA_TRY(cudaMemsetAsync(ms[i]->d_sticky, 0, sizeof(int), ms[i]->stream));
    }
    if (worst == 5) return fail(TNSIM_ETIMEOUT, "a bounded device wait ran out: an idle Jacobi CTA saw no progress or a tensor-core wait expired (step incomplete)");
    if (worst == 4) return fail(TNSIM_ENOCONV, "a Jacobi SVD reached max_sweeps (steps applied)");
    return TNSIM_OK;
}

tnsim_status tnsim_plan_create(tnsim_mps* const* ms, int32_t n_states, const int32_t* n2,
                               const int32_t* const* q_ptrs, const double* const* g4_dev,
                               const double* const* u1_dev, tnsim_plan** out) {
    if (!out) return fail(TNSIM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_states < 1 || !ms || !n2 || !q_ptrs || !g4_dev || !u1_dev) return fail(TNSIM_EINVAL, "bad arguments");
    for (int i = 0; i < n_states; ++i) {
        if (!ms[i]) return fail(TNSIM_EINVAL, "state is NULL");
        if (ms[i]->dt != ms[0]->dt || ms[i]->device != ms[0]->device || ms[i]->stream != ms[0]->stream ||
            ms[i]->p.gemm != ms[0]->p.gemm)
            return fail(TNSIM_EINVAL, "the states of a plan must share dtype, device, stream and gemm mode");
        for (int j = 0; j < i; ++j)
            if (ms[j] == ms[i]) return fail(TNSIM_EINVAL, "a state appears twice");
        tnsim_status st = check_pairs(ms[i], n2[i], q_ptrs[i]);
        if (st != TNSIM_OK) return st;
        if (n2[i] > 0 && !g4_dev[i]) return fail(TNSIM_EINVAL, "gate pointer is NULL");
    }
    tnsim_mps* m0 = ms[0];
    DevGuard g(m0->device);
    tnsim_plan* p = new (std::nothrow) tnsim_plan();
    if (!p) return fail(TNSIM_ENOMEM, "host allocation failed");
    p->states.assign(ms, ms + n_states);
    p->stream = m0->stream;
    p->device = m0->device;
    p->dt = m0->dt;
    p->gemm = m0->p.gemm;
    for (int i = 0; i < n_states; ++i) p->canon = p->canon || ms[i]->p.form == TNSIM_FORM_CANONICAL;
    p->jac_cfg = m0->jac_cfg;
    p->jac_spin = m0->jac_spin;
    for (int i = 0; i < n_states; ++i) p->qr = p->qr || (ms[i]->jac_cfg & 2) != 0;
    p->tc_mode = m0->tc_mode;
    p->tol = m0->p.jacobi_tol;
    std::vector<GateJob> jobs;
    std::vector<Site1Desc> s1;
    for (int i = 0; i < n_states; ++i) {
        tnsim_mps* m = ms[i];
        p->sweeps = std::max(p->sweeps, default_sweeps(m));
        std::vector<char> used(m->n, 0);
        for (int j = 0; j < n2[i]; ++j) {
            const int q = q_ptrs[i][j];
            used[q] = used[q + 1] = 1;
            GateJob jb;
            jb.m = m;
            jb.q = q;
            jb.slot = j;
            jb.g4 = g4_dev[i] + (size_t)j * 32;
            jb.uL = u1_dev[i] ? u1_dev[i] + (size_t)q * 8 : nullptr;
            jb.uR = u1_dev[i] ? u1_dev[i] + (size_t)(q + 1) * 8 : nullptr;
            jb.eps_dev = nullptr;
            jobs.push_back(jb);
            // launch shapes from the capacities: valid for any bond dimensions reached later
            p->chiL_max = std::max(p->chiL_max, m->cap[q]);
            p->chiM_max = std::max(p->chiM_max, m->cap[q + 1]);
            p->chiR_max = std::max(p->chiR_max, m->cap[q + 2]);
            p->k_max = std::max(p->k_max, m->cap[q + 1]);
        }
        if (u1_dev[i]) {
            for (int sidx = 0; sidx < m->n; ++sidx) {
                if (used[sidx]) continue;
                Site1Desc d;
                d.site = site_ptr(m, sidx);
                d.chi = m->d_chi;
                d.u = u1_dev[i] + (size_t)sidx * 8;
                d.q = sidx;
                d.pad_ = 0;
                s1.push_back(d);
                p->caplr = std::max(p->caplr, m->cap[sidx] * m->cap[sidx + 1]);
            }
        }
    }
    std::stable_sort(jobs.begin(), jobs.end(), [](const GateJob& a, const GateJob& b) {
        const double ca = (double)a.m->cap[a.q] * a.m->cap[a.q + 2] * a.m->cap[a.q + 2];
        const double cb = (double)b.m->cap[b.q] * b.m->cap[b.q + 2] * b.m->cap[b.q + 2];
        return ca > cb;
    });
    p->n_gates = (int)jobs.size();
    p->lead = leading_jobs(jobs, true);
    p->n_s1 = (int)s1.size();
    cudaError_t e = cudaMalloc((void**)&p->d_desc, sizeof(GateDesc) * (p->n_gates + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_out, sizeof(GateOut) * (p->n_gates + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_s1, sizeof(Site1Desc) * (p->n_s1 + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->d_ctl, sizeof(JacobiCtl));
    if (e != cudaSuccess) {
        cudaFree(p->d_desc); cudaFree(p->d_out); cudaFree(p->d_s1); cudaFree(p->d_ctl);
        delete p;
        return fail(TNSIM_ENOMEM, std::string("plan buffers: ") + cudaGetErrorString(e));
    }
    std::vector<GateDesc> hd(p->n_gates + 1);
    if (p->n_gates > 0) {
        tnsim_status st = upload_desc(p->stream, jobs, hd.data(), p->d_desc, p->d_out);
        if (st != TNSIM_OK) { tnsim_plan_destroy(p); return st; }
    }
    if (p->n_s1 > 0) e = cudaMemcpyAsync(p->d_s1, s1.data(), sizeof(Site1Desc) * p->n_s1, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) { tnsim_plan_destroy(p); return fail(TNSIM_ECUDA, cudaGetErrorString(e)); }
    *out = p;
    return TNSIM_OK;
}

tnsim_status tnsim_plan_launch(tnsim_plan* p) {
    if (!p) return fail(TNSIM_EINVAL, "plan is NULL");
    DevGuard g(p->device);
    cudaStream_t st = p->stream;
    if (p->n_s1 > 0) {
        CUDA_TRY(p->dt == TNSIM_C64 ? launch_site1q<float>(p->d_s1, p->n_s1, p->caplr, st)
                                    : launch_site1q<double>(p->d_s1, p->n_s1, p->caplr, st));
    }
    const int ng = p->n_gates;
    if (ng == 0) return TNSIM_OK;
    CUDA_TRY(cudaMemsetAsync(p->d_out, 0, sizeof(GateOut) * ng, st));
    CUDA_TRY(cudaMemsetAsync(p->d_ctl, 0, sizeof(JacobiCtl), st));
    const int m_max = 2 * p->chiL_max, n_max = 2 * p->chiR_max;
    if (p->dt == TNSIM_C128) {
        CUDA_TRY(launch_theta<double>(p->d_desc, ng, p->chiL_max, p->chiR_max, st));
        if (p->canon) CUDA_TRY(launch_scale_rows<double>(p->d_desc, ng, st));
        if (p->qr) CUDA_TRY(launch_qr<double>(p->d_desc, ng, m_max, st));
        CUDA_TRY(launch_jacobi<double>(p->d_desc, ng, m_max, n_max, p->tol, p->sweeps, p->d_ctl, st, p->jac_cfg,
                                       p->lead, p->jac_spin));
        CUDA_TRY(launch_truncate<double>(p->d_desc, ng, n_max, st));
        CUDA_TRY(launch_left<double>(p->d_desc, ng, m_max, p->k_max, st));
        CUDA_TRY(launch_right<double>(p->d_desc, ng, p->k_max, n_max, st));
        if (p->canon) CUDA_TRY(launch_left_canon<double>(p->d_desc, ng, m_max, p->k_max, st));
        if (p->qr) CUDA_TRY(launch_sites_pre<double>(p->d_desc, ng, m_max, p->k_max, n_max, st));
    } else {
        if (p->gemm == TNSIM_GEMM_FP32) CUDA_TRY(launch_theta<float>(p->d_desc, ng, p->chiL_max, p->chiR_max, st));
        else if (p->gemm == TNSIM_GEMM_FP32_3M) CUDA_TRY(launch_theta_3m(p->d_desc, ng, p->chiL_max, p->chiR_max, st));
        else CUDA_TRY(launch_theta_tc(p->tc_mode, p->d_desc, ng, p->chiL_max, p->chiM_max, p->chiR_max, st));
        if (p->canon) CUDA_TRY(launch_scale_rows<float>(p->d_desc, ng, st));
        if (p->qr) CUDA_TRY(launch_qr<float>(p->d_desc, ng, m_max, st));
        CUDA_TRY(launch_jacobi<float>(p->d_desc, ng, m_max, n_max, p->tol, p->sweeps, p->d_ctl, st, p->jac_cfg,
                                      p->lead, p->jac_spin));
        CUDA_TRY(launch_truncate<float>(p->d_desc, ng, n_max, st));
        CUDA_TRY(launch_left<float>(p->d_desc, ng, m_max, p->k_max, st));
        CUDA_TRY(launch_right<float>(p->d_desc, ng, p->k_max, n_max, st));
        if (p->canon) CUDA_TRY(launch_left_canon<float>(p->d_desc, ng, m_max, p->k_max, st));
        if (p->qr)
            CUDA_TRY(launch_sites_pre<float>(p->d_desc, ng, m_max, p->k_max, n_max, st,
                                             p->gemm == TNSIM_GEMM_TF32X3 || p->gemm == TNSIM_GEMM_BF16X3));
    }
    // the bond upper bounds the host keeps become the capacities
    for (tnsim_mps* m : p->states)
        for (int b = 0; b <= m->n; ++b) m->ub[b] = std::max(m->ub[b], m->cap[b]);
    return TNSIM_OK;
}

tnsim_status tnsim_plan_destroy(tnsim_plan* p) {
    if (!p) return TNSIM_OK;
    DevGuard g(p->device);
    cudaStreamSynchronize(p->stream);
    cudaFree(p->d_desc); cudaFree(p->d_out); cudaFree(p->d_s1); cudaFree(p->d_ctl);
    delete p;
    return TNSIM_OK;
}

tnsim_status tnsim_graph_create(tnsim_plan* const* plans, int32_t n_plans, tnsim_graph** out) {
    if (!out || !plans || n_plans < 1) return fail(TNSIM_EINVAL, "bad arguments");
    *out = nullptr;
    for (int i = 0; i < n_plans; ++i)
        if (!plans[i] || plans[i]->stream != plans[0]->stream) return fail(TNSIM_EINVAL, "plans must share a stream");
    DevGuard g(plans[0]->device);
    tnsim_graph* gr = new (std::nothrow) tnsim_graph();
    if (!gr) return fail(TNSIM_ENOMEM, "host allocation failed");
    gr->stream = plans[0]->stream;
    gr->device = plans[0]->device;
    if (gr->stream == nullptr) { delete gr; return fail(TNSIM_EINVAL, "graphs need a non-default stream"); }
    CUDA_TRY(cudaStreamSynchronize(gr->stream));
    cudaError_t e = cudaStreamBeginCapture(gr->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) { delete gr; return fail(TNSIM_ECUDA, std::string("capture: ") + cudaGetErrorString(e)); }
    tnsim_status st = TNSIM_OK;
    for (int i = 0; i < n_plans && st == TNSIM_OK; ++i) st = tnsim_plan_launch(plans[i]);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(gr->stream, &graph);
    if (st != TNSIM_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        delete gr;
        return st != TNSIM_OK ? st : fail(TNSIM_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    }
    gr->graph = graph;
    e = cudaGraphInstantiate(&gr->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete gr;
        return fail(TNSIM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    *out = gr;
    return TNSIM_OK;
}

tnsim_status tnsim_graph_launch(tnsim_graph* gr) {
    if (!gr) return fail(TNSIM_EINVAL, "graph is NULL");
    DevGuard g(gr->device);
    CUDA_TRY(cudaGraphLaunch(gr->exec, gr->stream));
    return TNSIM_OK;
}

tnsim_status tnsim_graph_destroy(tnsim_graph* gr) {
    if (!gr) return TNSIM_OK;
    DevGuard g(gr->device);
    cudaStreamSynchronize(gr->stream);
    if (gr->exec) cudaGraphExecDestroy(gr->exec);
    if (gr->graph) cudaGraphDestroy(gr->graph);
    delete gr;
    return TNSIM_OK;
}

tnsim_status tnsim_sync(tnsim_mps* m) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    DevGuard g(m->device);
    tnsim_status s = refresh_dims(m);
    if (s != TNSIM_OK) return s;
    int sticky = 0;
    CUDA_TRY(cudaMemcpy(&sticky, m->d_sticky, sizeof(int), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(m->d_sticky, 0, sizeof(int)));
    if (sticky == 5) return fail(TNSIM_ETIMEOUT, "a bounded device wait ran out: an idle Jacobi CTA saw no progress or a tensor-core wait expired (layer incomplete)");
    if (sticky) return fail(TNSIM_ENOCONV, "a Jacobi SVD reached max_sweeps (layer applied)");
    return TNSIM_OK;
}

tnsim_status tnsim_bond_dims(tnsim_mps* m, int32_t* out) {
    if (!m || !out) return fail(TNSIM_EINVAL, "NULL argument");
    DevGuard g(m->device);
    tnsim_status s = refresh_dims(m);
    if (s != TNSIM_OK) return s;
    for (int b = 0; b <= m->n; ++b) out[b] = m->ub[b];
    return TNSIM_OK;
}

tnsim_status tnsim_bond_spectrum(tnsim_mps* m, int32_t bond, double* s_out, int32_t* k_out) {
    if (!m || !s_out || !k_out) return fail(TNSIM_EINVAL, "NULL argument");
    if (bond < 0 || bond > m->n) return fail(TNSIM_EINVAL, "bond out of range");
    DevGuard g(m->device);
    CUDA_TRY(cudaStreamSynchronize(m->stream));
    int k = 0;
    CUDA_TRY(cudaMemcpy(&k, m->d_spec_k + bond, sizeof(int), cudaMemcpyDeviceToHost));
    *k_out = k;
    if (k > 0) CUDA_TRY(cudaMemcpy(s_out, m->d_spec + (size_t)bond * m->p.chi_max, sizeof(double) * k,
                                   cudaMemcpyDeviceToHost));
    return TNSIM_OK;
}

tnsim_status tnsim_export_sites(tnsim_mps* m, double* out, int64_t cap, int64_t* needed) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    DevGuard g(m->device);
    tnsim_status s = refresh_dims(m);
    if (s != TNSIM_OK) return s;
    int64_t need = 0;
    for (int q = 0; q < m->n; ++q) need += (int64_t)m->ub[q] * 2 * m->ub[q + 1] * 2;
    if (needed) *needed = need;
    if (!out) return TNSIM_OK;
    if (cap < need) return fail(TNSIM_EINVAL, "export buffer too small");
    std::vector<char> buf;
    int64_t pos = 0;
    for (int q = 0; q < m->n; ++q) {
        const size_t cnt = (size_t)m->ub[q] * 2 * m->ub[q + 1];
        buf.resize(cnt * m->esz);
        CUDA_TRY(cudaMemcpy(buf.data(), site_ptr(m, q), cnt * m->esz, cudaMemcpyDeviceToHost));
        if (m->dt == TNSIM_C64) {
            const float* f = (const float*)buf.data();
            for (size_t i = 0; i < 2 * cnt; ++i) out[pos + i] = (double)f[i];
        } else {
            std::memcpy(out + pos, buf.data(), cnt * 16);
        }
        pos += (int64_t)cnt * 2;
    }
    return TNSIM_OK;
}

tnsim_status tnsim_import_sites(tnsim_mps* m, const int32_t* dims, const double* data) {
    if (!m || !dims || !data) return fail(TNSIM_EINVAL, "NULL argument");
    if (m->p.form == TNSIM_FORM_CANONICAL)
        return fail(TNSIM_EUNSUPPORTED, "importing sites into a canonical-form state (its bond spectra are unknown)");
    if (dims[0] != 1 || dims[m->n] != 1) return fail(TNSIM_EINVAL, "terminal bonds must be 1");
    for (int b = 1; b < m->n; ++b)
        if (dims[b] < 1 || dims[b] > m->cap[b]) return fail(TNSIM_EINVAL, "bond dimension exceeds capacity");
    DevGuard g(m->device);
    CUDA_TRY(cudaStreamSynchronize(m->stream));
    std::vector<char> buf;
    int64_t pos = 0;
    for (int q = 0; q < m->n; ++q) {
        const size_t cnt = (size_t)dims[q] * 2 * dims[q + 1];
        if (!finite_all(data + pos, 2 * cnt)) return fail(TNSIM_EINVAL, "non-finite site entry");
        buf.resize(cnt * m->esz);
        if (m->dt == TNSIM_C64) {
            float* f = (float*)buf.data();
            for (size_t i = 0; i < 2 * cnt; ++i) f[i] = (float)data[pos + i];
        } else {
            std::memcpy(buf.data(), data + pos, cnt * 16);
        }
        CUDA_TRY(cudaMemcpy(site_ptr(m, q), buf.data(), cnt * m->esz, cudaMemcpyHostToDevice));
        pos += (int64_t)cnt * 2;
    }
    CUDA_TRY(cudaMemcpy(m->d_chi, dims, sizeof(int) * (m->n + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(m->d_spec_k, 0, sizeof(int) * (m->n + 1)));
    for (int b = 0; b <= m->n; ++b) m->ub[b] = dims[b];
    return TNSIM_OK;
}

tnsim_status tnsim_amplitudes(tnsim_mps* m, int64_t n_str, const uint8_t* bits, double* amps_out) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    if (n_str < 0) return fail(TNSIM_EINVAL, "n_str < 0");
    if (n_str == 0) return TNSIM_OK;
    if (!bits || !amps_out) return fail(TNSIM_EINVAL, "NULL argument");
    DevGuard g(m->device);
    tnsim_status s = refresh_dims(m);
    if (s != TNSIM_OK) return s;
    int chi_cap = 1;
    for (int b = 0; b <= m->n; ++b) chi_cap = std::max(chi_cap, m->ub[b]);
    const size_t nb = (size_t)n_str * m->n;
    void** d_sites = nullptr;
    uint8_t* d_bits = nullptr;
    double* d_amps = nullptr;
    std::vector<void*> ptrs(m->n);
    for (int q = 0; q < m->n; ++q) ptrs[q] = site_ptr(m, q);
    CUDA_TRY(cudaMalloc((void**)&d_sites, sizeof(void*) * m->n));
    cudaError_t e = cudaMalloc((void**)&d_bits, nb);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_amps, sizeof(double) * 2 * n_str);
    if (e == cudaSuccess) e = cudaMemcpy(d_sites, ptrs.data(), sizeof(void*) * m->n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_bits, bits, nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = (m->dt == TNSIM_C64)
                ? launch_amplitudes<float>(d_sites, m->d_chi, m->n, chi_cap, d_bits, n_str, d_amps, m->stream)
                : launch_amplitudes<double>(d_sites, m->d_chi, m->n, chi_cap, d_bits, n_str, d_amps, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e == cudaSuccess) e = cudaMemcpy(amps_out, d_amps, sizeof(double) * 2 * n_str, cudaMemcpyDeviceToHost);
    cudaFree(d_sites); cudaFree(d_bits); cudaFree(d_amps);
    if (e != cudaSuccess) return fail(TNSIM_ECUDA, std::string("amplitudes: ") + cudaGetErrorString(e));
    return TNSIM_OK;
}

tnsim_status tnsim_expect_pauli(tnsim_mps* m, int32_t n_terms, const char* paulis, double* out) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    if (n_terms < 0) return fail(TNSIM_EINVAL, "n_terms < 0");
    if (n_terms == 0) return TNSIM_OK;
    if (!paulis || !out) return fail(TNSIM_EINVAL, "NULL argument");
    const int n = m->n;
    for (int64_t i = 0; i < (int64_t)n_terms * n; ++i) {
        const char c = paulis[i];
        if (c != 'I' && c != 'X' && c != 'Y' && c != 'Z') return fail(TNSIM_EINVAL, "Pauli characters must be I, X, Y, Z");
    }
    DevGuard g(m->device);
    tnsim_status s = refresh_dims(m);
    if (s != TNSIM_OK) return s;
    int chi_cap = 1;
    for (int b = 0; b <= n; ++b) chi_cap = std::max(chi_cap, m->ub[b]);
    const size_t env = (size_t)chi_cap * chi_cap * m->esz;
    // operators: I, X, Y, Z as 2x2 complex128
    const double ops[4][8] = {{1, 0, 0, 0, 0, 0, 1, 0},
                              {0, 0, 1, 0, 1, 0, 0, 0},
                              {0, 0, 0, -1, 0, 1, 0, 0},
                              {1, 0, 0, 0, 0, 0, -1, 0}};
    char* d_L = nullptr; char* d_R = nullptr; char* d_tmp = nullptr; char* d_E = nullptr;
    double* d_ops = nullptr; double* d_res = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_L, env * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_R, env * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_tmp, env * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_E, env * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ops, sizeof(ops));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_res, sizeof(double) * 2 * n_terms);
    if (e == cudaSuccess) e = cudaMemcpy(d_ops, ops, sizeof(ops), cudaMemcpyHostToDevice);
    // identity boundary environments: L_0 = [[1]], R_n = [[1]]
    std::vector<char> one(m->esz, 0);
    if (m->dt == TNSIM_C64) { float f = 1.0f; std::memcpy(one.data(), &f, 4); }
    else { double f = 1.0; std::memcpy(one.data(), &f, 8); }
    if (e == cudaSuccess) e = cudaMemcpy(d_L, one.data(), m->esz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_R + env * n, one.data(), m->esz, cudaMemcpyHostToDevice);
    auto transfer = [&](int q, int op, const char* ein, char* eout, int left) -> cudaError_t {
        return (m->dt == TNSIM_C64)
                   ? launch_transfer<float>(site_ptr(m, q), m->d_chi, q, d_ops + 8 * op, ein, d_tmp, eout,
                                            chi_cap, left, m->stream)
                   : launch_transfer<double>(site_ptr(m, q), m->d_chi, q, d_ops + 8 * op, ein, d_tmp, eout,
                                             chi_cap, left, m->stream);
    };
    for (int q = 0; q < n && e == cudaSuccess; ++q) e = transfer(q, 0, d_L + env * q, d_L + env * (q + 1), 1);
    for (int q = n - 1; q >= 0 && e == cudaSuccess; --q) e = transfer(q, 0, d_R + env * (q + 1), d_R + env * q, 0);
    for (int t = 0; t < n_terms && e == cudaSuccess; ++t) {
        const char* ps = paulis + (size_t)t * n;
        int a = -1, b = -1;
        for (int q = 0; q < n; ++q)
            if (ps[q] != 'I') { if (a < 0) a = q; b = q; }
        auto opi = [](char c) { return c == 'I' ? 0 : c == 'X' ? 1 : c == 'Y' ? 2 : 3; };
        if (a < 0) {
            e = (m->dt == TNSIM_C64) ? launch_close<float>(d_L + env * n, d_R + env * n, m->d_chi, n, d_res + 2 * t, m->stream)
                                     : launch_close<double>(d_L + env * n, d_R + env * n, m->d_chi, n, d_res + 2 * t, m->stream);
            continue;
        }
        const char* cur = d_L + env * a;
        int pp = 0;
        for (int q = a; q <= b && e == cudaSuccess; ++q) {
            char* dst = d_E + env * pp;
            e = transfer(q, opi(ps[q]), cur, dst, 1);
            cur = dst;
            pp ^= 1;
        }
        if (e == cudaSuccess)
            e = (m->dt == TNSIM_C64) ? launch_close<float>(cur, d_R + env * (b + 1), m->d_chi, b + 1, d_res + 2 * t, m->stream)
                                     : launch_close<double>(cur, d_R + env * (b + 1), m->d_chi, b + 1, d_res + 2 * t, m->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e == cudaSuccess) e = cudaMemcpy(out, d_res, sizeof(double) * 2 * n_terms, cudaMemcpyDeviceToHost);
    cudaFree(d_L); cudaFree(d_R); cudaFree(d_tmp); cudaFree(d_E); cudaFree(d_ops); cudaFree(d_res);
    if (e != cudaSuccess) return fail(TNSIM_ECUDA, std::string("expect_pauli: ") + cudaGetErrorString(e));
    return TNSIM_OK;
}

tnsim_status tnsim_sample(tnsim_mps* m, int64_t n_shots, const double* uniforms, uint8_t* bits_out,
                          int64_t* n_nodes_out) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    if (n_shots < 0 || n_shots > (int64_t)1 << 24) return fail(TNSIM_EINVAL, "n_shots must be in [0, 2^24]");
    if (n_nodes_out) *n_nodes_out = 0;
    if (n_shots == 0) return TNSIM_OK;
    if (!uniforms || !bits_out) return fail(TNSIM_EINVAL, "NULL argument");
    const int n = m->n;
    const int64_t nu = n_shots * n;
    for (int64_t i = 0; i < nu; ++i)
        if (!(uniforms[i] >= 0.0 && uniforms[i] < 1.0)) return fail(TNSIM_EINVAL, "uniforms must lie in [0, 1)");
    DevGuard g(m->device);
    tnsim_status s = refresh_dims(m);   // exact bond dimensions on the host
    if (s != TNSIM_OK) return s;
    int chi_cap = 1;
    for (int b = 0; b <= n; ++b) chi_cap = std::max(chi_cap, m->ub[b]);
    const size_t es = m->esz, env = (size_t)chi_cap * chi_cap * es;
    const size_t S = (size_t)n_shots;
    cudaStream_t st = m->stream;
    // one stream-ordered allocation for everything
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_R = take(env * (n + 1)), o_tmp = take(env * 2), o_op = take(8 * sizeof(double));
    const size_t o_u = take(sizeof(double) * nu), o_bits = take((size_t)nu);
    const size_t o_v0 = take(S * chi_cap * es), o_v1 = take(S * chi_cap * es);
    const size_t o_w = take(S * 2 * chi_cap * es), o_y = take(S * 2 * chi_cap * es);
    const size_t o_p = take(sizeof(double) * 2 * S), o_flag = take(sizeof(int) * 2 * S);
    const size_t o_id = take(sizeof(int) * 2 * S), o_par = take(sizeof(int) * S), o_node = take(sizeof(int) * S);
    const size_t o_cnt = take(sizeof(int) + sizeof(unsigned long long) + 8);
    char* base = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&base, off, st));
    SampleWork w;
    w.v_cur = base + o_v0;
    w.v_next = base + o_v1;
    w.w = base + o_w;
    w.y = base + o_y;
    w.p = (double*)(base + o_p);
    w.flag = (int*)(base + o_flag);
    w.id = (int*)(base + o_id);
    w.parent = (int*)(base + o_par);
    w.node_of = (int*)(base + o_node);
    w.nodes = (int*)(base + o_cnt);
    w.total = (unsigned long long*)(base + o_cnt + 8);
    const double ident[8] = {1, 0, 0, 0, 0, 0, 1, 0};
    std::vector<char> one(es, 0);
    if (m->dt == TNSIM_C64) { const float f = 1.0f; std::memcpy(one.data(), &f, 4); }
    else { const double f = 1.0; std::memcpy(one.data(), &f, 8); }
    struct Cnt { int nodes; int pad; unsigned long long total; } c0 = {1, 0, 1ull};
    cudaError_t e = cudaMemcpyAsync(base + o_op, ident, sizeof(ident), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_u, uniforms, sizeof(double) * nu, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_R + env * n, one.data(), es, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_v0, one.data(), es, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_cnt, &c0, sizeof(c0), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.node_of, 0, sizeof(int) * S, st);
    // right environments R_n = [[1]], R_q from R_{q+1} (identity operator)
    for (int q = n - 1; q >= 1 && e == cudaSuccess; --q)
        e = (m->dt == TNSIM_C64)
                ? launch_transfer<float>(site_ptr(m, q), m->d_chi, q, (const double*)(base + o_op),
                                         base + o_R + env * (q + 1), base + o_tmp, base + o_R + env * q, chi_cap, 0, st)
                : launch_transfer<double>(site_ptr(m, q), m->d_chi, q, (const double*)(base + o_op),
                                          base + o_R + env * (q + 1), base + o_tmp, base + o_R + env * q, chi_cap, 0, st);
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
        const int64_t bound = q >= 40 ? n_shots : std::min<int64_t>(n_shots, (int64_t)1 << q);
        e = (m->dt == TNSIM_C64)
                ? launch_sample_site<float>(site_ptr(m, q), m->ub[q], m->ub[q + 1], base + o_R + env * (q + 1), q, n,
                                            n_shots, (int)bound, (const double*)(base + o_u), (uint8_t*)(base + o_bits), w, st)
                : launch_sample_site<double>(site_ptr(m, q), m->ub[q], m->ub[q + 1], base + o_R + env * (q + 1), q, n,
                                             n_shots, (int)bound, (const double*)(base + o_u), (uint8_t*)(base + o_bits), w, st);
        std::swap(w.v_cur, w.v_next);
    }
    Cnt c1 = {0, 0, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits_out, base + o_bits, (size_t)nu, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c1, base + o_cnt, sizeof(c1), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(base, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(TNSIM_ECUDA, std::string("sample: ") + cudaGetErrorString(e));
    // prefixes evaluated: every distinct prefix of length 0 .. n-1
    if (n_nodes_out) *n_nodes_out = (int64_t)c1.total - c1.nodes;
    return TNSIM_OK;
}

tnsim_status tnsim_set_wait_limits(tnsim_mps* m, int64_t jacobi_idle_polls, int64_t mbarrier_polls) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    if (jacobi_idle_polls < 0 || jacobi_idle_polls > 0xffffffffll || mbarrier_polls < 0 ||
        mbarrier_polls > 0x7fffffffll)
        return fail(TNSIM_EINVAL, "poll limits must be >= 0 and fit 32 bits");
    m->jac_spin = (unsigned)jacobi_idle_polls;
    m->tc_spin = (int)mbarrier_polls;
    return TNSIM_OK;
}

tnsim_status tnsim_set_device_memory_cap(int64_t bytes) {
    if (bytes < 0) return fail(TNSIM_EINVAL, "the cap must be >= 0 (0 = none)");
    g_dev_cap.store(bytes);
    return TNSIM_OK;
}

int64_t tnsim_device_bytes_held(void) { return g_dev_held.load(); }

tnsim_status tnsim_set_jacobi_config(tnsim_mps* m, int32_t cfg) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    if (cfg < 0 || cfg >= kJacobiConfigs) return fail(TNSIM_EINVAL, "unknown Jacobi configuration");
    m->jac_cfg = cfg;
    return TNSIM_OK;
}

tnsim_status tnsim_autotune(tnsim_mps* m, int32_t n2, const int32_t* q, const double* g4x4, int32_t reps,
                            int32_t* choice_out, double* ms_out) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    if (n2 < 1) return fail(TNSIM_EINVAL, "the tuning layer needs at least one gate");
    if (reps < 1 || reps > 100) return fail(TNSIM_EINVAL, "reps must be in [1, 100]");
    DevGuard g(m->device);
    tnsim_status s = check_pairs(m, n2, q);
    if (s != TNSIM_OK) return s;
    if (!g4x4 || !finite_all(g4x4, (size_t)n2 * 32)) return fail(TNSIM_EINVAL, "bad gate data");
    s = refresh_dims(m);   // exact bond dimensions: the tuned launches match real ones
    if (s != TNSIM_OK) return s;
    cudaStream_t st = m->stream;
    Staging* stg = acquire_staging(m);
    std::memcpy(stg->gates, g4x4, sizeof(double) * 32 * n2);
    CUDA_TRY(cudaMemcpyAsync(m->d_gates, stg->gates, sizeof(double) * 32 * n2, cudaMemcpyHostToDevice, st));
    std::vector<GateJob> jobs = layer_jobs(m, n2, q, m->d_gates, nullptr, nullptr);
    const int lead = leading_jobs(jobs, false);
    CUDA_TRY(cudaMemsetAsync(m->d_out, 0, sizeof(GateOut) * n2, st));
    s = upload_desc(st, jobs, stg->desc, m->d_desc, nullptr, 1);
    CUDA_TRY(cudaEventRecord(stg->done, st));
    if (s != TNSIM_OK) return s;
    int chiL_max = 1, chiM_max = 1, chiR_max = 1;
    for (const GateJob& j : jobs) {
        chiL_max = std::max(chiL_max, m->ub[j.q]);
        chiM_max = std::max(chiM_max, m->ub[j.q + 1]);
        chiR_max = std::max(chiR_max, m->ub[j.q + 2]);
    }
    const int m_max = 2 * chiL_max, n_max = 2 * chiR_max;
    // theta of every gate into the workspace (the sites are not touched)
    if (m->dt == TNSIM_C128 || m->p.gemm == TNSIM_GEMM_FP32) {
        CUDA_TRY(m->dt == TNSIM_C64 ? launch_theta<float>(m->d_desc, n2, chiL_max, chiR_max, st)
                                    : launch_theta<double>(m->d_desc, n2, chiL_max, chiR_max, st));
    } else if (m->p.gemm == TNSIM_GEMM_FP32_3M) {
        CUDA_TRY(launch_theta_3m(m->d_desc, n2, chiL_max, chiR_max, st));
    } else {
        CUDA_TRY(launch_theta_tc(m->tc_mode, m->d_desc, n2, chiL_max, chiM_max, chiR_max, st));
    }
    if (m->p.form == TNSIM_FORM_CANONICAL)
        CUDA_TRY(m->dt == TNSIM_C64 ? launch_scale_rows<float>(m->d_desc, n2, st)
                                    : launch_scale_rows<double>(m->d_desc, n2, st));
    // keep W and the gate records, restored before every timed launch
    const size_t wbytes = m->ws_elems * m->esz;
    char* bak = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&bak, (size_t)n2 * wbytes + sizeof(GateOut) * n2, st));
    for (int i = 0; i < n2; ++i)
        CUDA_TRY(cudaMemcpyAsync(bak + (size_t)i * wbytes, m->d_ws + ((size_t)i * 2 + 1) * wbytes, wbytes,
                                 cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(bak + (size_t)n2 * wbytes, m->d_out, sizeof(GateOut) * n2, cudaMemcpyDeviceToDevice, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    double best_ms = 0.0;
    int best = 0;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < kJacobiConfigs && e == cudaSuccess; ++c) {
        // configurations that launch the same kernels as an earlier one are not re-timed:
        // bit 0 with the tensor-core visits, and bit 2 for complex128 (no such path)
        const int same = (c & 4) ? (m->dt == TNSIM_C128 ? (c & 3) : ((c & 1) ? c - 1 : -1)) : -1;
        if (same >= 0) {
            if (ms_out) ms_out[c] = ms_out ? ms_out[same] : 0.0;
            continue;
        }
        double cmin = 0.0;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            for (int i = 0; i < n2 && e == cudaSuccess; ++i)
                e = cudaMemcpyAsync(m->d_ws + ((size_t)i * 2 + 1) * wbytes, bak + (size_t)i * wbytes, wbytes,
                                    cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(m->d_out, bak + (size_t)n2 * wbytes, sizeof(GateOut) * n2,
                                    cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(m->d_ctl, 0, sizeof(JacobiCtl), st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess && (c & 2))
                e = m->dt == TNSIM_C64 ? launch_qr<float>(m->d_desc, n2, m_max, st)
                                       : launch_qr<double>(m->d_desc, n2, m_max, st);
            if (e == cudaSuccess)
                e = m->dt == TNSIM_C64
                        ? launch_jacobi<float>(m->d_desc, n2, m_max, n_max, default_tol(m), default_sweeps(m), m->d_ctl, st, c,
                                               lead)
                        : launch_jacobi<double>(m->d_desc, n2, m_max, n_max, default_tol(m), default_sweeps(m), m->d_ctl, st, c,
                                                lead);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (r == 0 || ms < cmin)) cmin = ms;
        }
        if (ms_out) ms_out[c] = cmin;
        if (c == 0 || cmin < best_ms) { best_ms = cmin; best = c; }
    }
    cudaFreeAsync(bak, st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(TNSIM_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
    m->jac_cfg = best;
    if (choice_out) *choice_out = best;
    return TNSIM_OK;
}

tnsim_status tnsim_grad(const tnsim_circuit* c, const double* theta, const tnsim_hamiltonian* h, tnsim_dtype dt,
                        const tnsim_params* p, void* cuda_stream, double* energy_out, double* grad_out) {
    // ---- validation (nothing is allocated before it passes)
    if (!c || !theta || !h || !energy_out) return fail(TNSIM_EINVAL, "NULL argument");
    const int n = c->n_qubits, nl = c->n_layers;
    if (n < 2 || nl < 0) return fail(TNSIM_EINVAL, "bad circuit size");
    if (nl > 0 && (!c->n_rot || !c->n2)) return fail(TNSIM_EINVAL, "NULL layer arrays");
    if (dt != TNSIM_C64 && dt != TNSIM_C128) return fail(TNSIM_EINVAL, "unknown dtype");
    tnsim_params prm;
    tnsim_params_default(dt, &prm);
    if (p) prm = *p;
    tnsim_status s = check_params(&prm);
    if (s != TNSIM_OK) return s;
    if (prm.form != TNSIM_FORM_PAPER) return fail(TNSIM_EUNSUPPORTED, "tnsim_grad differentiates the paper's form only");
    std::vector<int64_t> rot_off(nl + 1, 0), gate_off(nl + 1, 0), ax_off(nl + 1, 0);
    for (int L = 0; L < nl; ++L) {
        if (c->n_rot[L] < 0 || c->n_rot[L] > 8) return fail(TNSIM_EINVAL, "n_rot must be in [0, 8]");
        if (c->n2[L] < 0 || c->n2[L] > n / 2) return fail(TNSIM_EINVAL, "bad pair count");
        ax_off[L + 1] = ax_off[L] + c->n_rot[L];
        rot_off[L + 1] = rot_off[L] + (int64_t)c->n_rot[L] * n;
        gate_off[L + 1] = gate_off[L] + c->n2[L];
    }
    if (ax_off[nl] > 0 && !c->axes) return fail(TNSIM_EINVAL, "NULL axes");
    for (int64_t i = 0; i < ax_off[nl]; ++i)
        if (c->axes[i] != 'X' && c->axes[i] != 'Y' && c->axes[i] != 'Z') return fail(TNSIM_EINVAL, "axes must be X, Y or Z");
    if (gate_off[nl] > 0 && (!c->q || !c->g4x4)) return fail(TNSIM_EINVAL, "NULL gate arrays");
    if (rot_off[nl] > 0 && !grad_out) return fail(TNSIM_EINVAL, "grad_out is NULL");
    for (int L = 0; L < nl; ++L) {
        std::vector<char> used(n, 0);
        for (int64_t i = gate_off[L]; i < gate_off[L + 1]; ++i) {
            const int q = c->q[i];
            if (q < 0 || q >= n - 1 || used[q] || used[q + 1]) return fail(TNSIM_EINVAL, "bad or overlapping pair");
            used[q] = used[q + 1] = 1;
        }
    }
    if (!finite_all(c->g4x4, (size_t)gate_off[nl] * 32) || !finite_all(theta, (size_t)rot_off[nl]))
        return fail(TNSIM_EINVAL, "non-finite gate entry or angle");
    if (h->n_terms < 1 || !h->paulis || !h->coeffs) return fail(TNSIM_EINVAL, "empty Hamiltonian");
    struct Term { int a, b; double coef; int idx; };
    std::vector<Term> terms;
    double id_coef = 0.0;
    for (int t = 0; t < h->n_terms; ++t) {
        int a = -1, b = -1;
        for (int q = 0; q < n; ++q) {
            const char ch = h->paulis[(size_t)t * n + q];
            if (ch != 'I' && ch != 'X' && ch != 'Y' && ch != 'Z') return fail(TNSIM_EINVAL, "Pauli characters must be I, X, Y, Z");
            if (ch != 'I') { if (a < 0) a = q; b = q; }
        }
        if (!std::isfinite(h->coeffs[t])) return fail(TNSIM_EINVAL, "non-finite coefficient");
        if (a < 0) id_coef += h->coeffs[t];
        else terms.push_back({a, b, h->coeffs[t], t});
    }
    // ---- a state of our own on the caller's stream
    tnsim_mps* m = nullptr;
    s = tnsim_mps_create(n, dt, &prm, cuda_stream, &m);
    if (s != TNSIM_OK) return s;
    struct Guard { tnsim_mps* m; std::vector<void*> bufs;
        ~Guard() { if (m) cudaStreamSynchronize(m->stream); for (void* b : bufs) cudaFree(b); if (m) tnsim_mps_destroy(m); } } gd{m, {}};
    DevGuard dg(m->device);
    cudaStream_t st = m->stream;
    const size_t es = m->esz, AB = m->arena_bytes;
    int cap_max = 1;
    for (int b = 0; b <= n; ++b) cap_max = std::max(cap_max, m->cap[b]);
    const size_t env = (size_t)cap_max * cap_max * es;
    const size_t cm = 2 * (size_t)m->capmax;
    auto dalloc = [&](size_t bytes) -> char* {
        void* ptr = nullptr;
        if (cudaMalloc(&ptr, std::max<size_t>(bytes, 256)) != cudaSuccess) return nullptr;
        gd.bufs.push_back(ptr);
        return (char*)ptr;
    };
    const int64_t n_theta = rot_off[nl];
    const int64_t n_gates_all = gate_off[nl];
    char* d_theta = dalloc(sizeof(double) * std::max<int64_t>(n_theta, 1));
    char* d_axes = dalloc(std::max<int64_t>(ax_off[nl], 1));
    double* d_u1 = (double*)dalloc(sizeof(double) * 8 * (size_t)std::max<int64_t>(n_theta, 1) * 1);
    double* d_ubar = (double*)dalloc(sizeof(double) * 8 * (size_t)std::max<int64_t>(n_theta, 1) + sizeof(double) * 16 * m->G);
    double* d_grad = (double*)dalloc(sizeof(double) * std::max<int64_t>(n_theta, 1));
    double* d_g4 = (double*)dalloc(sizeof(double) * 32 * std::max<int64_t>(n_gates_all, 1));
    RotLayer* d_rl = (RotLayer*)dalloc(sizeof(RotLayer) * std::max(nl, 1));
    char* d_ckpt = dalloc((AB + sizeof(int) * (n + 1) + 255) / 256 * 256 * (size_t)(nl + 1));
    char* d_env = dalloc(env * (size_t)(4 * (n + 1) + 4) + env * 2 * terms.size());
    char* d_adj = dalloc(AB * 4);
    char* d_scr = dalloc(9 * cm * cm * es * (size_t)m->G);
    GradGateDesc* d_gdesc = (GradGateDesc*)dalloc(sizeof(GradGateDesc) * m->G);
    Site1Bwd* d_s1 = (Site1Bwd*)dalloc(sizeof(Site1Bwd) * n);
    double* d_ops = (double*)dalloc(sizeof(double) * 32);
    if (!d_theta || !d_axes || !d_u1 || !d_ubar || !d_grad || !d_g4 || !d_rl || !d_ckpt || !d_env || !d_adj || !d_scr ||
        !d_gdesc || !d_s1 || !d_ops)
        return fail(TNSIM_ENOMEM, "tnsim_grad: device allocation failed");
    // one 2x2 gate per (layer with rotations, qubit)
    std::vector<int64_t> u1_off(nl, -1);
    int64_t u1n = 0;
    for (int L = 0; L < nl; ++L)
        if (c->n_rot[L] > 0) { u1_off[L] = u1n; u1n += (int64_t)n * 8; }
    std::vector<RotLayer> rl(std::max(nl, 1));
    for (int L = 0; L < nl; ++L) {
        rl[L].axes = d_axes + ax_off[L];
        rl[L].theta = (const double*)d_theta + rot_off[L];
        rl[L].n_rot = c->n_rot[L];
        rl[L].pad_ = 0;
        rl[L].u1_off = std::max<int64_t>(u1_off[L], 0);
        rl[L].grad_off = rot_off[L];
    }
    const double ops[4][8] = {{1, 0, 0, 0, 0, 0, 1, 0}, {0, 0, 1, 0, 1, 0, 0, 0},
                              {0, 0, 0, -1, 0, 1, 0, 0}, {1, 0, 0, 0, 0, 0, -1, 0}};
    auto opi = [](char ch) { return ch == 'I' ? 0 : ch == 'X' ? 1 : ch == 'Y' ? 2 : 3; };
    CUDA_TRY(cudaMemcpyAsync(d_ops, ops, sizeof(ops), cudaMemcpyHostToDevice, st));
    if (n_theta > 0) CUDA_TRY(cudaMemcpyAsync(d_theta, theta, sizeof(double) * n_theta, cudaMemcpyHostToDevice, st));
    if (ax_off[nl] > 0) CUDA_TRY(cudaMemcpyAsync(d_axes, c->axes, ax_off[nl], cudaMemcpyHostToDevice, st));
    if (n_gates_all > 0) CUDA_TRY(cudaMemcpyAsync(d_g4, c->g4x4, sizeof(double) * 32 * n_gates_all, cudaMemcpyHostToDevice, st));
    if (nl > 0) CUDA_TRY(cudaMemcpyAsync(d_rl, rl.data(), sizeof(RotLayer) * nl, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(d_ubar, 0, sizeof(double) * 8 * (size_t)std::max<int64_t>(n_theta, 1) + sizeof(double) * 16 * m->G, st));
    if (nl > 0) CUDA_TRY(launch_rot_build(d_rl, nl, n, d_u1, st));
    // every checkpoint starts on a 256-byte boundary (its sites are read with 16-byte accesses)
    const size_t ck_stride = (AB + sizeof(int) * (n + 1) + 255) / 256 * 256;
    auto ck_sites = [&](int L) { return d_ckpt + ck_stride * (size_t)L; };
    auto ck_chi = [&](int L) { return (int*)(d_ckpt + ck_stride * (size_t)L + AB); };
    auto layer_u1 = [&](int L) -> const double* { return c->n_rot[L] > 0 ? d_u1 + u1_off[L] : nullptr; };
    auto run_layer = [&](int L) -> tnsim_status {
        Staging* stg = acquire_staging(m);
        tnsim_status r = enqueue_layer(m, stg, c->n2[L], c->q + gate_off[L], d_g4 + gate_off[L] * 32, layer_u1(L), nullptr);
        cudaEventRecord(stg->done, st);
        return r;
    };
    // ---- forward with a checkpoint before every layer (and of the final state)
    for (int L = 0; L <= nl; ++L) {
        CUDA_TRY(cudaMemcpyAsync(ck_sites(L), m->d_sites, AB, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(ck_chi(L), m->d_chi, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, st));
        if (L < nl) {
            s = run_layer(L);
            if (s != TNSIM_OK) return s;
        }
    }
    std::vector<int> chi_h((size_t)(nl + 1) * (n + 1));
    for (int L = 0; L <= nl; ++L)
        CUDA_TRY(cudaMemcpyAsync(chi_h.data() + (size_t)L * (n + 1), ck_chi(L), sizeof(int) * (n + 1),
                                 cudaMemcpyDeviceToHost, st));
    int sticky = 0;
    CUDA_TRY(cudaMemcpyAsync(&sticky, m->d_sticky, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (sticky == 5) return fail(TNSIM_ETIMEOUT, "a bounded device wait ran out: an idle Jacobi CTA saw no progress or a tensor-core wait expired (forward incomplete)");
    auto chi_at = [&](int L, int b) { return chi_h[(size_t)L * (n + 1) + b]; };
    // ---- energy and the adjoint of the final state (environments of the final state)
    const int* dchi = m->d_chi;   // the final bond dimensions
    char* L0 = d_env;
    char* R0 = L0 + env * (n + 1);
    char* LH = R0 + env * (n + 1);
    char* RH = LH + env * (n + 1);
    char* tmp = RH + env * (n + 1);            // 2 env
    char* part = tmp + env * 2;                // 2 env (running partial)
    char* full = part + env * 2;               // 2 env per term (left full, right full)
    char* AH = d_adj;                          // adjoint of <H> (arena layout)
    char* AN = d_adj + AB;                     // adjoint of the norm
    char* ABc = d_adj + 2 * AB;                // adjoint of the current (post-layer) state
    char* ABn = d_adj + 3 * AB;
    std::vector<char> one(es, 0);
    if (dt == TNSIM_C64) { const float f = 1.0f; std::memcpy(one.data(), &f, 4); }
    else { const double f = 1.0; std::memcpy(one.data(), &f, 8); }
    CUDA_TRY(cudaMemsetAsync(d_env, 0, env * (size_t)(4 * (n + 1) + 4) + env * 2 * terms.size(), st));
    CUDA_TRY(cudaMemsetAsync(d_adj, 0, AB * 4, st));
    CUDA_TRY(cudaMemcpyAsync(L0, one.data(), es, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(R0 + env * n, one.data(), es, cudaMemcpyHostToDevice, st));
    const bool c64 = dt == TNSIM_C64;
    auto transfer = [&](int q, const double* op, const char* ein, char* eout, int left) -> cudaError_t {
        return c64 ? launch_transfer<float>(site_ptr(m, q), dchi, q, op, ein, tmp, eout, cap_max, left, st)
                   : launch_transfer<double>(site_ptr(m, q), dchi, q, op, ein, tmp, eout, cap_max, left, st);
    };
    auto site_adj = [&](int q, const char* E, const double* op, const char* Rt, double coef, char* out) -> cudaError_t {
        cudaError_t e = c64 ? launch_apply_rt<float>(site_ptr(m, q), dchi, q, Rt, tmp, cap_max, st)
                            : launch_apply_rt<double>(site_ptr(m, q), dchi, q, Rt, tmp, cap_max, st);
        if (e != cudaSuccess) return e;
        return c64 ? launch_site_adj2<float>(E, op, tmp, dchi, q, coef, out + m->site_off[q], cap_max, st)
                   : launch_site_adj2<double>(E, op, tmp, dchi, q, coef, out + m->site_off[q], cap_max, st);
    };
    auto axpy = [&](char* dst, const char* src, int bond, double coef, int zero_first) -> cudaError_t {
        return c64 ? launch_env_axpy<float>(dst, src, dchi, bond, coef, zero_first, cap_max, st)
                   : launch_env_axpy<double>(dst, src, dchi, bond, coef, zero_first, cap_max, st);
    };
    const double* opI = d_ops;
    for (int q = 0; q < n; ++q) CUDA_TRY(transfer(q, opI, L0 + env * q, L0 + env * (q + 1), 1));
    for (int q = n - 1; q >= 0; --q) CUDA_TRY(transfer(q, opI, R0 + env * (q + 1), R0 + env * q, 0));
    // every non-identity term: the sites it covers, and its full left / right environments
    for (size_t t = 0; t < terms.size(); ++t) {
        const Term& tm = terms[t];
        const char* ps = h->paulis + (size_t)tm.idx * n;
        char* Lfull = full + env * 2 * t;
        char* Rfull = Lfull + env;
        // every site of the support: left partial over a..q-1, right partial over q+1..b
        // (recomputed per site; Pauli supports are short)
        for (int q = tm.a; q <= tm.b; ++q) {
            // left partial over a..q-1 into part[0]
            CUDA_TRY(cudaMemcpyAsync(part, L0 + env * tm.a, env, cudaMemcpyDeviceToDevice, st));
            for (int x = tm.a; x < q; ++x) {
                CUDA_TRY(transfer(x, d_ops + 8 * opi(ps[x]), part, part + env, 1));
                CUDA_TRY(cudaMemcpyAsync(part, part + env, env, cudaMemcpyDeviceToDevice, st));
            }
            // right partial over q+1..b into Rfull (scratch)
            CUDA_TRY(cudaMemcpyAsync(Rfull, R0 + env * (tm.b + 1), env, cudaMemcpyDeviceToDevice, st));
            for (int x = tm.b; x > q; --x) {
                CUDA_TRY(transfer(x, d_ops + 8 * opi(ps[x]), Rfull, part + env, 0));
                CUDA_TRY(cudaMemcpyAsync(Rfull, part + env, env, cudaMemcpyDeviceToDevice, st));
            }
            CUDA_TRY(site_adj(q, part, d_ops + 8 * opi(ps[q]), Rfull, tm.coef, AH));
        }
        // full environments of the term
        CUDA_TRY(cudaMemcpyAsync(Lfull, L0 + env * tm.a, env, cudaMemcpyDeviceToDevice, st));
        for (int x = tm.a; x <= tm.b; ++x) {
            CUDA_TRY(transfer(x, d_ops + 8 * opi(ps[x]), Lfull, part, 1));
            CUDA_TRY(cudaMemcpyAsync(Lfull, part, env, cudaMemcpyDeviceToDevice, st));
        }
        CUDA_TRY(cudaMemcpyAsync(Rfull, R0 + env * (tm.b + 1), env, cudaMemcpyDeviceToDevice, st));
        for (int x = tm.b; x >= tm.a; --x) {
            CUDA_TRY(transfer(x, d_ops + 8 * opi(ps[x]), Rfull, part, 0));
            CUDA_TRY(cudaMemcpyAsync(Rfull, part, env, cudaMemcpyDeviceToDevice, st));
        }
    }
    // LH[q]: terms entirely left of bond q; RH[q]: terms entirely right of it
    CUDA_TRY(axpy(LH, L0, 0, id_coef, 1));
    for (int q = 0; q < n; ++q) {
        CUDA_TRY(transfer(q, opI, LH + env * q, LH + env * (q + 1), 1));
        for (size_t t = 0; t < terms.size(); ++t)
            if (terms[t].b == q) CUDA_TRY(axpy(LH + env * (q + 1), full + env * 2 * t, q + 1, terms[t].coef, 0));
    }
    for (int q = n - 1; q >= 0; --q) {
        CUDA_TRY(transfer(q, opI, RH + env * (q + 1), RH + env * q, 0));
        for (size_t t = 0; t < terms.size(); ++t)
            if (terms[t].a == q) CUDA_TRY(axpy(RH + env * q, full + env * 2 * t + env, q, terms[t].coef, 0));
    }
    for (int q = 0; q < n; ++q) {
        CUDA_TRY(site_adj(q, LH + env * q, opI, R0 + env * (q + 1), 1.0, AH));
        CUDA_TRY(site_adj(q, L0 + env * q, opI, RH + env * (q + 1), 1.0, AH));
        CUDA_TRY(site_adj(q, L0 + env * q, opI, R0 + env * (q + 1), 1.0, AN));
    }
    // energy = LH[n] / L0[n]
    double hs[2] = {0, 0}, nr[2] = {0, 0};
    if (c64) {
        float a2[2], b2[2];
        CUDA_TRY(cudaMemcpyAsync(a2, LH + env * n, 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(b2, L0 + env * n, 8, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        hs[0] = a2[0]; nr[0] = b2[0];
    } else {
        CUDA_TRY(cudaMemcpyAsync(hs, LH + env * n, 16, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(nr, L0 + env * n, 16, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    *energy_out = hs[0] / nr[0];
    const int64_t arena_elems = (int64_t)(AB / es);
    CUDA_TRY(c64 ? launch_adj_combine<float>(AH, AN, LH + env * n, L0 + env * n, arena_elems, st)
                 : launch_adj_combine<double>(AH, AN, LH + env * n, L0 + env * n, arena_elems, st));
    CUDA_TRY(cudaMemcpyAsync(ABc, AH, AB, cudaMemcpyDeviceToDevice, st));
    // ---- backward, layer by layer: restore, recompute, differentiate every gate
    std::vector<GradGateDesc> hg(m->G);
    std::vector<Site1Bwd> hs1(n);
    for (int L = nl - 1; L >= 0; --L) {
        CUDA_TRY(cudaMemcpyAsync(m->d_sites, ck_sites(L), AB, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(m->d_chi, ck_chi(L), sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, st));
        for (int b = 0; b <= n; ++b) m->ub[b] = chi_at(L, b);
        s = run_layer(L);
        if (s != TNSIM_OK) return s;
        CUDA_TRY(cudaMemsetAsync(ABn, 0, AB, st));
        const int n2 = c->n2[L];
        const int32_t* ql = c->q + gate_off[L];
        const double* u1 = layer_u1(L);
        std::vector<char> paired(n, 0);
        for (int i = 0; i < n2; ++i) {
            const int q = ql[i];
            paired[q] = paired[q + 1] = 1;
            GradGateDesc& d = hg[i];
            std::memset(&d, 0, sizeof(d));
            char* ws = m->d_ws + (size_t)i * 2 * m->ws_elems * es;
            d.a_pre = ck_sites(L) + m->site_off[q];
            d.b_pre = ck_sites(L) + m->site_off[q + 1];
            d.u_post = ck_sites(L + 1) + m->site_off[q];
            d.y_post = ck_sites(L + 1) + m->site_off[q + 1];
            d.theta0 = ws;
            d.W = ws + m->ws_elems * es;
            d.s2 = m->d_s2 + (size_t)i * 2 * m->capmax;
            d.perm = m->d_perm + (size_t)i * 2 * m->capmax;
            d.g4 = d_g4 + (gate_off[L] + i) * 32;
            d.uL = u1 ? u1 + (size_t)q * 8 : nullptr;
            d.uR = u1 ? u1 + (size_t)(q + 1) * 8 : nullptr;
            d.ub_post = ABc + m->site_off[q];
            d.bb_post = ABc + m->site_off[q + 1];
            d.ab_pre = ABn + m->site_off[q];
            d.bb_pre = ABn + m->site_off[q + 1];
            double* ub0 = u1 ? d_ubar + u1_off[L] : d_ubar + (size_t)8 * std::max<int64_t>(n_theta, 1);
            d.ubar_l = u1 ? ub0 + (size_t)q * 8 : ub0 + (size_t)i * 16;
            d.ubar_r = u1 ? ub0 + (size_t)(q + 1) * 8 : ub0 + (size_t)i * 16 + 8;
            d.scratch = d_scr + (size_t)i * 9 * cm * cm * es;
            d.chiL = chi_at(L, q);
            d.chiM = chi_at(L, q + 1);
            d.chiR = chi_at(L, q + 2);
            d.k = chi_at(L + 1, q + 1);
            d.renorm = prm.renormalize ? 1 : 0;
            d.cm = (int)cm;
        }
        if (n2 > 0) {
            CUDA_TRY(cudaMemcpyAsync(d_gdesc, hg.data(), sizeof(GradGateDesc) * n2, cudaMemcpyHostToDevice, st));
            CUDA_TRY(c64 ? launch_gate_bwd<float>(d_gdesc, n2, st) : launch_gate_bwd<double>(d_gdesc, n2, st));
        }
        int ns = 0;
        for (int q = 0; q < n; ++q) {
            if (paired[q]) continue;
            const size_t bytes = (size_t)chi_at(L, q) * 2 * chi_at(L, q + 1) * es;
            if (!u1) {
                CUDA_TRY(cudaMemcpyAsync(ABn + m->site_off[q], ABc + m->site_off[q], bytes, cudaMemcpyDeviceToDevice, st));
                continue;
            }
            Site1Bwd& d = hs1[ns++];
            d.ab_post = ABc + m->site_off[q];
            d.a_pre = ck_sites(L) + m->site_off[q];
            d.ab_pre = ABn + m->site_off[q];
            d.u = u1 + (size_t)q * 8;
            d.ubar = d_ubar + u1_off[L] + (size_t)q * 8;
            d.cl = chi_at(L, q);
            d.cr = chi_at(L, q + 1);
        }
        if (ns > 0) {
            CUDA_TRY(cudaMemcpyAsync(d_s1, hs1.data(), sizeof(Site1Bwd) * ns, cudaMemcpyHostToDevice, st));
            CUDA_TRY(c64 ? launch_site1_bwd<float>(d_s1, ns, st) : launch_site1_bwd<double>(d_s1, ns, st));
        }
        // the host arrays above are read by the copies before the next layer reuses them
        CUDA_TRY(cudaStreamSynchronize(st));
        std::swap(ABc, ABn);
    }
    if (n_theta > 0) {
        CUDA_TRY(launch_rot_grad(d_rl, nl, n, d_ubar, d_grad, st));
        CUDA_TRY(cudaMemcpyAsync(grad_out, d_grad, sizeof(double) * n_theta, cudaMemcpyDeviceToHost, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    return TNSIM_OK;
}

tnsim_status tnsim_last_stats(tnsim_mps* m, tnsim_stats* out) {
    if (!m || !out) return fail(TNSIM_EINVAL, "NULL argument");
    DevGuard g(m->device);
    CUDA_TRY(cudaStreamSynchronize(m->stream));
    unsigned long long st[9];
    static_assert(sizeof(st) == sizeof(tnsim_stats), "one device counter per tnsim_stats field");
    CUDA_TRY(cudaMemcpy(st, m->d_stats, sizeof(st), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemset(m->d_stats, 0, sizeof(st)));
    out->gates = (int64_t)st[0];
    out->sweeps = (int64_t)st[1];
    out->rotations = (int64_t)st[2];
    out->pair_visits = (int64_t)st[3];
    out->visit_rows = (int64_t)st[4];
    out->rotation_rows = (int64_t)st[5];
    out->theta_cmacs = (int64_t)st[6];
    out->right_cmacs = (int64_t)st[7];
    out->qr_cmacs = (int64_t)st[8];
    return TNSIM_OK;
}

tnsim_status tnsim_profile_enable(tnsim_mps* m, int32_t on) {
    if (!m) return fail(TNSIM_EINVAL, "state is NULL");
    DevGuard g(m->device);
    if (!on) {
        CUDA_TRY(cudaStreamSynchronize(m->stream));
        for (auto& r : m->recs) { m->ev_pool.push_back(r.a); m->ev_pool.push_back(r.b); }
        m->recs.clear();
    }
    m->prof_on = on != 0;
    return TNSIM_OK;
}

tnsim_status tnsim_profile_read(tnsim_mps* m, double* ms, int64_t* launches) {
    if (!m || !ms || !launches) return fail(TNSIM_EINVAL, "NULL argument");
    DevGuard g(m->device);
    CUDA_TRY(cudaStreamSynchronize(m->stream));
    for (int i = 0; i < TNSIM_K_COUNT; ++i) { ms[i] = 0.0; launches[i] = 0; }
    for (auto& r : m->recs) {
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.cls] += t;
        launches[r.cls] += 1;
        m->ev_pool.push_back(r.a);
        m->ev_pool.push_back(r.b);
    }
    m->recs.clear();
    return TNSIM_OK;
}

}  // extern "C"

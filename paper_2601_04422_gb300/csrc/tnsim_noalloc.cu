// One two-qubit update that allocates no memory (tnsim_two_site_update_noalloc).
//
// Some callers cannot let a library call cudaMalloc: a plugin running inside an
// application whose memory pool owns the whole device, a process that works under
// a fixed device-memory budget, or a loop that must not synchronise the device
// (cudaMalloc and cudaFree may synchronise).  This entry point runs the same
// kernels as tnsim_apply_layer for a single pair, but all of its scratch (the
// theta and Jacobi working matrices, the sorted spectrum, the gate descriptor and
// counters) lives in one fixed array compiled into the library.
//
// That array is a file-scope __device__ variable: every GPU that loads the library
// holds it (about 1.1 MB) until the process exits.  On the host its name is only a
// stand-in, so its device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on it.
// Every call shares the array and leaves the previous call's contents in it; the
// parts that must start at zero are cleared on the stream before each use.  Two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and give wrong results.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/tnsim.h"
#include "tnsim_internal.h"

using namespace tnsim;

namespace {

constexpr int kNaMaxDim = 256;                       // m = 2 chi_L, n = 2 chi_R, k, chi_max
constexpr size_t kNaMat = (size_t)kNaMaxDim * kNaMaxDim * sizeof(float2);

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t al(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t OFF_DESC = 0;
constexpr size_t OFF_OUT = al(OFF_DESC + sizeof(GateDesc));
constexpr size_t OFF_CHI = al(OFF_OUT + sizeof(GateOut));              // 3 ints
constexpr size_t OFF_SMALL = al(OFF_CHI + 4 * sizeof(int));            // spec_k, sticky
constexpr size_t OFF_STATS = al(OFF_SMALL + 4 * sizeof(int));          // 8 u64
constexpr size_t OFF_CTL = al(OFF_STATS + 8 * sizeof(unsigned long long));
constexpr size_t OFF_G4 = al(OFF_CTL + sizeof(JacobiCtl));
constexpr size_t OFF_EPS = al(OFF_G4 + 32 * sizeof(double));
constexpr size_t OFF_S2 = al(OFF_EPS + sizeof(double));
constexpr size_t OFF_PERM = al(OFF_S2 + kNaMaxDim * sizeof(double));
constexpr size_t OFF_SPEC = al(OFF_PERM + kNaMaxDim * sizeof(int));
constexpr size_t OFF_THETA = al(OFF_SPEC + kNaMaxDim * sizeof(double));
constexpr size_t OFF_W = al(OFF_THETA + kNaMat);
constexpr size_t NA_BYTES = al(OFF_W + kNaMat);

}  // namespace

// The scratch array itself (device memory of every GPU that loads the library).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

std::mutex g_na_mu;
constexpr int kNaMaxDevices = 64;
char* g_na_ptr[kNaMaxDevices] = {};

tnsim_status na_fail(tnsim_status s, const std::string& m) {
    tnsim::set_last_error(m.c_str());   // read back through tnsim_last_error()
    return s;
}

}  // namespace

extern "C" tnsim_status tnsim_two_site_update_noalloc(
    void* site_a, int64_t cap_a, void* site_b, int64_t cap_b, int32_t chi_l, int32_t chi_m,
    int32_t chi_r, const double* g4x4, int32_t chi_max, double cutoff, int32_t renormalize,
    void* cuda_stream, int32_t* k_out, double* eps_out, double* s_out) {
    tnsim::set_last_error("");
    if (!site_a || !site_b || !g4x4 || !k_out) return na_fail(TNSIM_EINVAL, "NULL argument");
    if (chi_l < 1 || chi_m < 1 || chi_r < 1) return na_fail(TNSIM_EINVAL, "bond dimensions must be >= 1");
    if (2 * chi_l > kNaMaxDim || 2 * chi_r > kNaMaxDim)
        return na_fail(TNSIM_EINVAL, "chi_l and chi_r must be <= 128: the fixed scratch holds "
                                     "matrices of at most 256 x 256");
    if (chi_max < 1 || chi_max > kNaMaxDim) return na_fail(TNSIM_EINVAL, "chi_max must be in [1, 256]");
    if (!(cutoff >= 0.0 && cutoff < 1.0)) return na_fail(TNSIM_EINVAL, "cutoff must be in [0, 1)");
    const int kcap = std::min(chi_max, std::min(2 * chi_l, 2 * chi_r));
    const int64_t bond = std::max(chi_m, kcap);
    if (cap_a < (int64_t)chi_l * 2 * bond || cap_b < bond * 2 * (int64_t)chi_r)
        return na_fail(TNSIM_EINVAL, "site capacity too small for the input or the kept bond");
    for (int i = 0; i < 32; ++i)
        if (!std::isfinite(g4x4[i])) return na_fail(TNSIM_EINVAL, "non-finite gate entry");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(TNSIM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices) return na_fail(TNSIM_EUNSUPPORTED, "device index too large");
    char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(TNSIM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_ptr[dev] = (char*)p;
        }
        base = g_na_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;

    GateDesc d;
    std::memset(&d, 0, sizeof(d));
    d.siteA = site_a;
    d.siteB = site_b;
    d.chi = (int*)(base + OFF_CHI);
    d.g4 = (const double*)(base + OFF_G4);
    d.theta0 = base + OFF_THETA;
    d.W = base + OFF_W;
    d.s2 = (double*)(base + OFF_S2);
    d.perm = (int*)(base + OFF_PERM);
    d.spectrum = (double*)(base + OFF_SPEC);
    d.spec_k = (int*)(base + OFF_SMALL);
    d.eps_out = (double*)(base + OFF_EPS);
    d.out = (GateOut*)(base + OFF_OUT);
    d.sticky = (int*)(base + OFF_SMALL) + 1;
    d.stats = (unsigned long long*)(base + OFF_STATS);
    d.cutoff = cutoff;
    d.q = 0;
    d.chi_max = chi_max;
    d.renorm = renormalize ? 1 : 0;
    const int chi[3] = {chi_l, chi_m, chi_r};

#define NA_TRY(call)                                                                     \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return na_fail(TNSIM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

    NA_TRY(cudaMemcpyAsync(base + OFF_DESC, &d, sizeof(d), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(base + OFF_CHI, chi, sizeof(chi), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(base + OFF_G4, g4x4, 32 * sizeof(double), cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemsetAsync(base + OFF_OUT, 0, sizeof(GateOut), st));
    NA_TRY(cudaMemsetAsync(base + OFF_SMALL, 0, 4 * sizeof(int), st));
    NA_TRY(cudaMemsetAsync(base + OFF_STATS, 0, 8 * sizeof(unsigned long long), st));
    NA_TRY(cudaMemsetAsync(base + OFF_CTL, 0, sizeof(JacobiCtl), st));
    const GateDesc* dd = (const GateDesc*)(base + OFF_DESC);
    NA_TRY(launch_theta<float>(dd, 1, chi_l, chi_r, st));
    NA_TRY(launch_jacobi<float>(dd, 1, 2 * chi_l, 2 * chi_r, 0.0, 40, (JacobiCtl*)(base + OFF_CTL), st));
    NA_TRY(launch_truncate<float>(dd, 1, 2 * chi_r, st));
    NA_TRY(launch_left<float>(dd, 1, 2 * chi_l, kcap, st));
    NA_TRY(launch_right<float>(dd, 1, kcap, 2 * chi_r, st));
    GateOut o;
    NA_TRY(cudaMemcpyAsync(&o, base + OFF_OUT, sizeof(o), cudaMemcpyDeviceToHost, st));
    // the kept count is known only after the sync: copy every entry that can be kept
    // (k <= kcap) on the caller's stream, then clear the ones past k on the host
    if (s_out) NA_TRY(cudaMemcpyAsync(s_out, base + OFF_SPEC, sizeof(double) * kcap, cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    *k_out = o.k;
    if (eps_out) *eps_out = o.eps;
    if (s_out)
        for (int j = std::max(o.k, 0); j < chi_max; ++j) s_out[j] = 0.0;
#undef NA_TRY
    if (o.status == 5) return na_fail(TNSIM_ETIMEOUT, "the Jacobi kernel saw no progress (update incomplete)");
    if (o.status) return na_fail(TNSIM_ENOCONV, "the Jacobi SVD reached its sweep cap (update applied)");
    return TNSIM_OK;
}

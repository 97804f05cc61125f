// Host planner for gate lists: non-local two-qubit gates through SWAP chains, and
// layerization into layers of disjoint nearest-neighbour pairs (Sec. IV.B).
//
// A two-qubit gate on qubits (a, b) with |a - b| > 1 is made local the way the
// paper's SWAP method does it: the far qubit b is moved next to a by SWAP gates on
// neighbouring pairs, the gate acts on the now-adjacent pair, and the same SWAPs
// in reverse order put every qubit back in place.  Each SWAP is an ordinary
// two-qubit update (merge, gate, truncated SVD, absorb), so it can truncate.
//
// The resulting stream of local operations is then cut into layers with the
// as-soon-as-possible rule: an operation goes to the first layer after the last
// layer that holds a two-qubit gate on one of its qubits.  A one-qubit gate may
// share a layer with a later two-qubit gate on the same qubit because a layer
// applies its one-qubit gates first (on paired qubits they are multiplied into the
// 4x4 on the device); consecutive one-qubit gates on a qubit are multiplied on the
// host.  Operations on disjoint qubits commute exactly -- a two-qubit update reads
// and writes only its own two sites and their shared bond -- so running the layers
// gives the same state as running the list in order, truncation included.
//
// Pure host code: no CUDA call is made here.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "tnsim_circuit.h"
#include "tnsim_internal.h"

namespace tnsim {

namespace {

// 4x4 complex (row-major, interleaved) with the two qubits of its basis index
// exchanged: G'[(2y+x),(2y'+x')] = G[(2x+y),(2x'+y')].
void swap_qubit_order(const double* g, double* out) {
    auto idx = [](int s) { return ((s & 1) << 1) | (s >> 1); };
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            const int rs = idx(r), cs = idx(c);
            out[2 * (4 * r + c)] = g[2 * (4 * rs + cs)];
            out[2 * (4 * r + c) + 1] = g[2 * (4 * rs + cs) + 1];
        }
}

// out = u * v for 2x2 complex (row-major, interleaved); out may alias neither
void mul2(const double* u, const double* v, double* out) {
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double re = 0, im = 0;
            for (int k = 0; k < 2; ++k) {
                const double ar = u[2 * (2 * r + k)], ai = u[2 * (2 * r + k) + 1];
                const double br = v[2 * (2 * k + c)], bi = v[2 * (2 * k + c) + 1];
                re += ar * br - ai * bi;
                im += ar * bi + ai * br;
            }
            out[2 * (2 * r + c)] = re;
            out[2 * (2 * r + c) + 1] = im;
        }
}

// SWAP in the basis 2 b_q + b_{q+1}: |01> <-> |10>, |00> and |11> fixed
void swap_gate(double* g) {
    std::memset(g, 0, sizeof(double) * 32);
    const int map[4] = {0, 2, 1, 3};
    for (int r = 0; r < 4; ++r) g[2 * (4 * r + map[r])] = 1.0;
}

struct LocalOp {
    int q;           // first qubit (the pair is (q, q+1) for two-qubit operations)
    bool two;        // two-qubit operation
    double m[32];    // 4x4 (two) or 2x2 in the first 8 doubles
};

}  // namespace

tnsim_status layerize_circuit(int n, int n_ops, const int32_t* qa, const int32_t* qb, const double* mats,
                              CircuitLayers& out, std::string& err) {
    out = CircuitLayers();
    out.n = n;
    if (n < 2) { err = "n_qubits must be >= 2"; return TNSIM_EINVAL; }
    if (n_ops < 0) { err = "n_ops must be >= 0"; return TNSIM_EINVAL; }
    if (n_ops > 0 && (!qa || !qb || !mats)) { err = "NULL operation array"; return TNSIM_EINVAL; }
    // expand into local operations
    std::vector<LocalOp> ops;
    ops.reserve((size_t)n_ops);
    for (int i = 0; i < n_ops; ++i) {
        const int a = qa[i], b = qb[i];
        const double* g = mats + (size_t)i * 32;
        if (a < 0 || a >= n) { err = "operation " + std::to_string(i) + ": qubit out of range"; return TNSIM_EINVAL; }
        const int nval = b < 0 ? 8 : 32;
        for (int k = 0; k < nval; ++k)
            if (!std::isfinite(g[k])) { err = "operation " + std::to_string(i) + ": non-finite entry"; return TNSIM_EINVAL; }
        LocalOp op;
        std::memset(&op, 0, sizeof(op));
        if (b < 0) {
            op.q = a;
            op.two = false;
            std::memcpy(op.m, g, sizeof(double) * 8);
            ops.push_back(op);
            continue;
        }
        if (b >= n || b == a) { err = "operation " + std::to_string(i) + ": bad second qubit"; return TNSIM_EINVAL; }
        // the pair in increasing order, with the gate's basis index to match
        int lo = a, hi = b;
        double gl[32];
        if (a < b) std::memcpy(gl, g, sizeof(gl));
        else { swap_qubit_order(g, gl); lo = b; hi = a; }
        LocalOp sw;
        std::memset(&sw, 0, sizeof(sw));
        sw.two = true;
        swap_gate(sw.m);
        // move qubit hi down to lo + 1
        for (int j = hi - 1; j > lo; --j) { sw.q = j; ops.push_back(sw); }
        op.q = lo;
        op.two = true;
        std::memcpy(op.m, gl, sizeof(gl));
        ops.push_back(op);
        // and back
        for (int j = lo + 1; j < hi; ++j) { sw.q = j; ops.push_back(sw); }
    }
    // as-soon-as-possible layers
    std::vector<int> last2(n, -1), last1(n, -1);
    std::vector<std::vector<int>> lq;         // pairs per layer
    std::vector<std::vector<double>> lg;      // 32 doubles per pair
    std::vector<std::vector<double>> lu;      // n * 8 doubles, identity where unused
    std::vector<char> lhas;
    auto ensure = [&](int L) {
        while ((int)lq.size() <= L) {
            lq.emplace_back();
            lg.emplace_back();
            std::vector<double> u((size_t)n * 8, 0.0);
            for (int x = 0; x < n; ++x) { u[(size_t)x * 8 + 0] = 1.0; u[(size_t)x * 8 + 6] = 1.0; }
            lu.push_back(std::move(u));
            lhas.push_back(0);
        }
    };
    for (const LocalOp& op : ops) {
        if (!op.two) {
            const int x = op.q;
            const int L = std::max(last2[x] + 1, last1[x]);
            ensure(L);
            double* u = lu[L].data() + (size_t)x * 8;
            double prod[8];
            mul2(op.m, u, prod);      // the new gate acts after the ones already in the slot
            std::memcpy(u, prod, sizeof(prod));
            lhas[L] = 1;
            last1[x] = L;
        } else {
            const int x = op.q;
            const int L = std::max({last2[x] + 1, last2[x + 1] + 1, last1[x], last1[x + 1], 0});
            ensure(L);
            lq[L].push_back(x);
            lg[L].insert(lg[L].end(), op.m, op.m + 32);
            last2[x] = last2[x + 1] = L;
        }
    }
    const int nl = (int)lq.size();
    out.n2.resize(nl);
    out.q_off.resize(nl + 1, 0);
    out.has_u1.resize(nl);
    for (int L = 0; L < nl; ++L) {
        out.n2[L] = (int)lq[L].size();
        out.q_off[L + 1] = out.q_off[L] + out.n2[L];
        out.has_u1[L] = lhas[L];
        out.q.insert(out.q.end(), lq[L].begin(), lq[L].end());
        out.g4.insert(out.g4.end(), lg[L].begin(), lg[L].end());
        out.u1.insert(out.u1.end(), lu[L].begin(), lu[L].end());
    }
    return TNSIM_OK;
}

}  // namespace tnsim

extern "C" tnsim_status tnsim_circuit_layerize(int32_t n_qubits, int32_t n_ops, const int32_t* qa,
                                               const int32_t* qb, const double* mats, int32_t cap_layers,
                                               int32_t cap_gates, int32_t* n_layers, int32_t* n_gates,
                                               int32_t* layer_n2, int32_t* gate_q, double* gate_g4,
                                               double* layer_u1) {
    tnsim::set_last_error("");
    if (!n_layers || !n_gates) {
        tnsim::set_last_error("n_layers and n_gates must not be NULL");
        return TNSIM_EINVAL;
    }
    tnsim::CircuitLayers cl;
    std::string err;
    tnsim_status s = tnsim::layerize_circuit(n_qubits, n_ops, qa, qb, mats, cl, err);
    if (s != TNSIM_OK) {
        tnsim::set_last_error(err.c_str());
        return s;
    }
    *n_layers = (int32_t)cl.n2.size();
    *n_gates = (int32_t)cl.q.size();
    if (!layer_n2 && !gate_q && !gate_g4 && !layer_u1) return TNSIM_OK;   // sizes only
    if (cap_layers < *n_layers || cap_gates < *n_gates || !layer_n2 || !gate_q || !gate_g4 || !layer_u1) {
        tnsim::set_last_error("output capacity too small (n_layers / n_gates hold the sizes needed)");
        return TNSIM_EINVAL;
    }
    for (size_t L = 0; L < cl.n2.size(); ++L) layer_n2[L] = cl.n2[L];
    std::memcpy(gate_q, cl.q.data(), sizeof(int32_t) * cl.q.size());
    std::memcpy(gate_g4, cl.g4.data(), sizeof(double) * cl.g4.size());
    std::memcpy(layer_u1, cl.u1.data(), sizeof(double) * cl.u1.size());
    return TNSIM_OK;
}

// Host planner of gate lists (tnsim_circuit.cu): SWAP chains for non-local gates
// and as-soon-as-possible layers of disjoint nearest-neighbour pairs (Sec. IV.B).
#pragma once

#include <string>
#include <vector>

#include "../../include/tnsim.h"

namespace tnsim {

// Layers of a gate list.  Layer L holds n2[L] pairs (q[q_off[L] + i], +1) with
// their 4x4 gates (32 doubles each, g4[32 * (q_off[L] + i) ...]) and n one-qubit
// gates (u1[8 n L ...], identity where none), applied before the pairs; has_u1[L]
// says whether any of them differs from the identity.
struct CircuitLayers {
    int n = 0;
    std::vector<int> n2, q_off, q;
    std::vector<char> has_u1;
    std::vector<double> g4, u1;
};

// Expand and layerize n_ops operations: (qa[i], qb[i]) with qb[i] < 0 for a one-qubit
// gate (2x2 in the first 8 doubles of mats[32 i ...]), else a two-qubit gate on any
// two distinct qubits, 4x4 in the basis 2 b_qa + b_qb.  Host only.
tnsim_status layerize_circuit(int n, int n_ops, const int32_t* qa, const int32_t* qb, const double* mats,
                              CircuitLayers& out, std::string& err);

}  // namespace tnsim

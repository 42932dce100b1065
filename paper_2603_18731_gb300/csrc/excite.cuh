// Excitation-driven evaluation of ladder groups (fermionic operators).
#pragma once

#include "apply_kernel.cuh"

namespace qsd {

constexpr int kMaxShapes = 16;

// A ladder term is nonzero at row r only if the row is occupied on the term's
// raising qubits and empty on its lowering qubits.  Its shape counts these per
// sector (sector 0 = qubits [0, split), sector 1 = [split, n)):
//   bits 0-3: occupied in sector 0, 4-7: empty in sector 0,
//   bits 8-11: occupied in sector 1, 12-15: empty in sector 1.
struct ExcParams {
    HashView ght;             // flip mask -> excitation-group index
    const int32_t *exc_gid;   // [G_exc] group index of each excitation group
    const int32_t *dense;     // rank index (nullptr: use ght): entry -> group or -1
    uint32_t dbase[kMaxShapes], dstride[kMaxShapes];  // per shape: signature base, C(n1, b1)
    const int32_t *rest_gid;  // [G_rest] groups evaluated by the per-row scan
    int64_t n_rest;
    int split;
    int n_qubits;
    int n_shapes;
    uint32_t shapes[kMaxShapes];
};

// Launch the warp-per-row excitation product for precision mode PREC.
template <int PREC>
void launch_apply_exc(const ApplyParams &p, const ExcParams &e, int W, int KB, cudaStream_t s);

}  // namespace qsd

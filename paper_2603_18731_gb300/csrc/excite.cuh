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

// The masks of one term and its phase side by side (whole 16-byte loads), for
// the factored product (W <= 2).  Two arrays: in one, q is the phase in
// 64-bit fixed point, q = phi 2^e rounded to an integer, with one exponent e
// per operator chosen so that any group's sum of |q| stays below 2^62 (a sum
// of terms is then an exact integer sum, converted to FP64 once); in the
// other, q holds the bits of the FP64 phase.
template <int W> struct TermRec;
template <> struct alignas(16) TermRec<1> {
    uint64_t P[1], V[1], Z[1];
    int64_t q;
};
template <> struct alignas(16) TermRec<2> {
    uint64_t P[2], V[2], Z[2];
    int64_t q;
    uint64_t pad;
};

template <int W>
__device__ __forceinline__ TermRec<W> load_term(const TermRec<W> *__restrict__ r) {
    static_assert(sizeof(TermRec<W>) % 16 == 0, "whole 16-byte loads");
    TermRec<W> out;
    const uint4 *src = reinterpret_cast<const uint4 *>(r);
    uint4 *dst = reinterpret_cast<uint4 *>(&out);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(TermRec<W>) / 16); ++i) dst[i] = __ldg(src + i);
    return out;
}

// Launch the warp-per-row excitation product for precision mode PREC.
template <int PREC>
void launch_apply_exc(const ApplyParams &p, const ExcParams &e, int W, int KB, cudaStream_t s);

}  // namespace qsd

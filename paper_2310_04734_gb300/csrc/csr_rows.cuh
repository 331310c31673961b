// Row-group traversal of the CSR model (K, D, M share one pattern) for the FP64
// sparse products: the residual r = f - A(w) x (paper Sec. 3.3, Eq. 8), the GMRES
// operator, the moment recurrences (Eq. 9/10) and the projection products
// A V (Sec. 3.3, Galerkin projection).
//
// A group of kRowLanes consecutive lanes owns one row; lane g takes the entries
// rowptr[i] + g, + g + kRowLanes, ... so the group reads each run of values and
// column indices as one contiguous segment (coalesced 16-byte loads of K and D),
// and the partial sums are combined by shuffles inside the group (a reduce-scatter
// when a row carries several load columns).  The number of columns is a template
// parameter: with a runtime count the compiler predicates the unused columns' DFMAs,
// which still occupy the FP64 pipe.  Rows are
// walked by a CTA-uniform loop, so every lane of a warp takes part in every
// shuffle.  On GB300 these kernels are bound by the FP64 pipe (~1.25 TFLOP/s,
// one 64th of the FP32 rate), not by HBM: a complex multiply-add costs 4 DFMA
// per 16-byte operand, so the entry formation is kept to 3 DFMA per entry and
// the fluid/shell scale tests run on the integer pipe.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"

namespace fsi {

constexpr int kRowLanes = 4;                     // lanes per row group
static_assert(kRowLanes == 4, "the three-product kernel of the greedy relies on one slot per lane");
constexpr int kRowThreads = 256;                 // threads per CTA of the row-group kernels
constexpr int kRowsPerCta = kRowThreads / kRowLanes;

// sum over the kRowLanes lanes of a group (all lanes of the warp must call it)
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int off = kRowLanes / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ double2 group_sum(double2 v) { return make_double2(group_sum(v.x), group_sum(v.y)); }

__device__ __forceinline__ double shfl_x(double v, int d) { return __shfl_xor_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double2 shfl_x(double2 v, int d) { return make_double2(shfl_x(v.x, d), shfl_x(v.y, d)); }
__device__ __forceinline__ double add_(double a, double b) { return a + b; }
__device__ __forceinline__ double2 add_(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Reduce-scatter of S partial sums (S a power of two) over the lanes of a group: each
// halving step sends half of the held slots to the partner lane and adds the other half,
// so a lane pays S/2 + S/4 + ... additions instead of S per step of a full all-reduce.
// Afterwards lane g holds the group totals of slots slot_base<S>(g) + q, q < kept_slots<S>.
template <int S>
__host__ __device__ constexpr int kept_slots() { return S > kRowLanes ? S / kRowLanes : 1; }
template <int S>
__device__ __forceinline__ int slot_base(int g) {
    return S >= kRowLanes ? g * (S / kRowLanes) : g / (kRowLanes / S);
}
// lanes that hold a distinct set of slots (one per duplicate set when S < kRowLanes)
template <int S>
__device__ __forceinline__ bool slot_writer(int g) {
    return S >= kRowLanes ? true : (g % (kRowLanes / S)) == 0;
}
template <int S, typename T>
__device__ __forceinline__ void group_reduce_scatter(T (&v)[S], int g) {
    static_assert((S & (S - 1)) == 0 && S >= 1, "power-of-two slot count");
    int held = S;
#pragma unroll
    for (int d = kRowLanes / 2; d >= 1; d >>= 1) {
        if (held > 1) {
            const int h = held / 2;
            const bool upper = (g & d) != 0;
#pragma unroll
            for (int q = 0; q < S / 2; ++q)
                if (q < h) {
                    const T keep = upper ? v[q + h] : v[q];
                    const T send = upper ? v[q] : v[q + h];
                    v[q] = add_(keep, shfl_x(send, d));
                }
            held = h;
        } else {
            v[0] = add_(v[0], shfl_x(v[0], d));
        }
    }
}

// A(w)_e = K_e + i w D_e - w^2 M_e with w2 = w * w precomputed (3 DFMA)
__device__ __forceinline__ double2 a_entry_ld(const DevModel& m, int64_t e, double w, double w2) {
    const double2 k = __ldg(m.K + e), d = __ldg(m.D + e);
    const double mm = __ldg(m.M + e);
    return make_double2(fma(-w2, mm, fma(-w, d.y, k.x)), fma(w, d.x, k.y));
}

inline int device_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// CTAs of `kernel` (kRowThreads threads, no dynamic shared memory) resident per SM
template <typename Kern>
int resident_ctas(Kern kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRowThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm;
}

// grid.x of a row-group kernel launched with F frequency (or column) slices in grid.y:
// one full wave of CTAs over all SMs in total (per_sm resident CTAs each), each CTA
// walking several row blocks
inline unsigned row_grid_x(int64_t n, int F, int per_sm) {
    const int64_t blocks = (n + kRowsPerCta - 1) / kRowsPerCta;
    const int64_t ctas = int64_t(device_sms()) * per_sm;
    int64_t want = (ctas + F - 1) / (F > 0 ? F : 1);
    if (want < 1) want = 1;
    return unsigned(want < blocks ? want : blocks);
}

}  // namespace fsi

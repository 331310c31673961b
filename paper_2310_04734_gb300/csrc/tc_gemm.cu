// Trailing updates of the band LU on the 5th-generation tensor cores (tcgen05),
// with operands and results moved by the Tensor Memory Accelerator (TMA).
//
//   C[r0:r1, c0:c1] -= A[r0:r1, k0:k0+K] * B[k0:k0+K, c0:c1]      (complex FP32, row major)
//
// The complex product is one real GEMM on interleaved storage: with A' the
// M x 2K real view of A and B' the 2K x 2N real matrix with 2x2 blocks
// [[Br, Bi], [-Bi, Br]], C' -= A' B' is exactly the complex update on the
// interleaved C (four real products per complex multiply-add).
//
// Precision.  These factors precondition systems with condition numbers up to
// ~1e8, and the refinement converges only if the factor is about as accurate
// as an FP32 one.  Two properties of the tensor pipe stand in the way and are
// handled here:
//   * products: every FP32 operand is split into three BF16 planes,
//     x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1),
//     24 significant bits in all), and six products are accumulated:
//     a0 b0 into a "big" accumulator, a0 b1 + a1 b0 + a0 b2 + a2 b0 + a1 b1
//     into a "small" one; the terms left out are below 2^-24 relative (adding
//     a1 b2 + a2 b1 changed neither the GMRES steps nor the time on config 2).
//     (Three TF32 products, hi/lo splits of 11 bits each, keep only ~22 bits
//     and needed about twice the GMRES steps of an FP32 factor.)
//   * accumulation: the tensor core adds into its FP32 accumulator without
//     rounding to nearest, so long sums drift; measured on config 2, K = 852
//     complex in one accumulation needed four times the GMRES steps.  Here
//     each "big" accumulation spans 32 elements of K only: it is
//     double-buffered in TMEM (2 x 128 columns), and the epilogue warps drain
//     each one into FP32 registers (round to nearest) while the MMAs of the
//     next one run.  The "small" sums are 2^-8 of the big ones, so the same
//     truncation per add costs 2^-8 as much: they accumulate over the whole
//     K of a tile (double-buffered per tile, 2 x 128 columns) and are drained
//     once, at the end of the tile (measured on config 2: the same GMRES
//     steps as draining them with the big sums, 5.5 % less kernel time).
// With one plane (NP = 1) the same kernel computes the plain BF16 product
// a0 b0 (FP32 accumulation), the low-precision factor of the mixed-precision
// study, which the FP64 refinement has to make up for.
//
// Two kernels per update:
//   pack:  A' and B' are split into NP BF16 planes in K-major layout (rows of
//          Kp elements, Kp = 2K rounded up to 64, zero padded): A' rows are
//          the rows of C, B' rows are the real columns of C (B transposed).
//   gemm:  one CTA per 128 x 128 real tile of C and frequency, warp
//          specialised: warp 0 issues the TMA loads of the 2 NP operand tiles
//          of a 64-element K slice (128-byte swizzle), warp 1 issues the
//          tcgen05.mma instructions (M = N = 128, K = 16, kind::f16 with BF16
//          operands) and commits them per slice, warps 4..7 drain the TMEM
//          accumulators with tcgen05.ld into register sums and finally add
//          -sum into C with TMA bulk reductions (cp.reduce.async.bulk.tensor
//          .add), which also drop the rows and columns outside C.
// Every mbarrier wait is bounded by a spin limit (a kernel argument): on a
// timeout the CTA records an error, stops issuing work, waits (with a fixed
// generous limit) for the TMA loads and MMAs it already issued, and only then
// frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>

#include "kernels.cuh"
#include "prof.h"

namespace fsi {

namespace {

constexpr int kTM = 128;             // real rows per tile (MMA M)
constexpr int kTN = 128;             // real columns per tile (MMA N)
constexpr int kTK = 64;              // BF16 elements per K slice: one 128-byte swizzle row
constexpr int kThreads = 256;
constexpr int kTmemCols = 512;       // big sums: 2 x 128 fp32 columns; small sums: 2 x 128
constexpr int kPlaneBytes = 128 * 128;   // one 128-row plane of a slice (A and B alike)
// Each poll of an mbarrier may suspend the thread for up to kPollNs (it resumes as soon as the
// phase completes); a wait gives up after `limit` polls, so the default bounds a wait by ~17 s.
// Measured on a probe of the update's MMA pattern: waits with this hint issue the next MMAs 8 %
// sooner than polls without one.
constexpr uint32_t kPollNs = 4000;
constexpr uint32_t kDefaultSpin = 1u << 22;
constexpr uint32_t kDrainSpin = 1u << 22;   // waits for work already issued (always completes)

constexpr int kStagingBytes = 4 * 2 * 4096;   // output staging: 4 drain warps x 2 buffers

template <int NP>
struct Cfg {
    static constexpr int kStageBytes = 2 * NP * kPlaneBytes;          // NP planes of A and of B
    static constexpr int kStages = NP == 3 ? 2 : 4;
    static constexpr size_t kSmem = size_t(kStages) * kStageBytes + kStagingBytes + 1024 + 256;
};

std::atomic<uint32_t> g_spin_limit{kDefaultSpin};

// K steps of 16 accumulated in TMEM between drains: 2 (32 elements).  Measured on config 2,
// batch 96: 5.45 GMRES steps and 32.2 frequencies/s, against 5.67 and 31.1 with 4 steps (64
// elements) and 5.38 and 28.7 with 1 step.
constexpr int kDrainKSteps = 2;
int drain_ksteps() { return kDrainKSteps; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// x = x0 + x1 + x2 in BF16 (each remainder is exact in FP32)
template <int NP>
__device__ __forceinline__ void split(float x, __nv_bfloat16 (&p)[NP]) {
    p[0] = __float2bfloat16_rn(x);
    if constexpr (NP == 3) {
        const float r1 = x - __bfloat162float(p[0]);
        p[1] = __float2bfloat16_rn(r1);
        p[2] = __float2bfloat16_rn(r1 - __bfloat162float(p[1]));
    }
}

// ----------------------------------------------------------------- operand packing
// Ap[NP f + p][r][kk] = plane p of A'[r0 + r][2 k0 + kk] for kk < 2K, 0 up to Kp.
template <int NP>
__global__ void pack_a_kernel(const float* __restrict__ G, int64_t sGf, int64_t ldf, int r0, int M, int kx0, int K2,
                              int Kp, __nv_bfloat16* __restrict__ Ap) {
    const int f = blockIdx.y;
    const int64_t idx = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) * 8;
    const int64_t plane = int64_t(M) * Kp;
    if (idx >= plane) return;
    const int r = int(idx / Kp), kk = int(idx - int64_t(r) * Kp);
    const float* src = G + f * sGf + int64_t(r0 + r) * ldf + kx0;
    __align__(16) __nv_bfloat16 out[NP][8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        __nv_bfloat16 p[NP];
        split<NP>((kk + j < K2) ? src[kk + j] : 0.f, p);
#pragma unroll
        for (int q = 0; q < NP; ++q) out[q][j] = p[q];
    }
#pragma unroll
    for (int q = 0; q < NP; ++q)
        *reinterpret_cast<uint4*>(Ap + (int64_t(NP) * f + q) * plane + idx) = *reinterpret_cast<const uint4*>(out[q]);
}

// Bp[NP f + p][q][kk0 + kk]: row q = 2n holds (Br, -Bi) and row 2n + 1 holds (Bi, Br) of
// every complex k < kfill (at kk = 2k, 2k + 1), zero for K <= k; B[k][n] = G[k0 + k][c0 + n];
// rows of `pitch` elements.
template <int NP>
__global__ void pack_b_kernel(const float2* __restrict__ G, int64_t sG, int ld, int k0, int K, int c0, int N,
                              int pitch, int kk0, int kfill, __nv_bfloat16* __restrict__ Bp) {
    __shared__ float2 t[32][33];
    const int f = blockIdx.z;
    const int kb = blockIdx.x * 32, nb = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float2* Gf = G + f * sG;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = kb + ty + 8 * i, n = nb + tx;
        t[ty + 8 * i][tx] = (k < K && n < N) ? Gf[int64_t(k0 + k) * ld + c0 + n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int64_t plane = int64_t(2 * N) * pitch;
    const int k = kb + tx;
    if (k >= kfill) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int nl = ty + 8 * i, n = nb + nl;
        if (n >= N) continue;
        const float2 b = t[tx][nl];
        const int64_t o0 = int64_t(2 * n) * pitch + kk0 + 2 * k, o1 = o0 + pitch;
        __nv_bfloat16 re[NP], mi[NP], im[NP];
        split<NP>(b.x, re);
        split<NP>(-b.y, mi);
        split<NP>(b.y, im);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            __nv_bfloat16* P = Bp + (int64_t(NP) * f + q) * plane;
            __nv_bfloat162 v0, v1;
            v0.x = re[q];
            v0.y = mi[q];
            v1.x = im[q];
            v1.y = re[q];
            *reinterpret_cast<__nv_bfloat162*>(P + o0) = v0;
            *reinterpret_cast<__nv_bfloat162*>(P + o1) = v1;
        }
    }
}

// ----------------------------------------------------------------- tcgen05 / TMA helpers
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFFu) >> 4);          // start address
    d |= uint64_t(1024u >> 4) << 32;                // stride byte offset
    d |= uint64_t(1) << 46;                         // descriptor version
    d |= uint64_t(2) << 61;                         // 128-byte swizzle
    return d;
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(kTN >> 3) << 17) | (uint32_t(kTM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint32_t a, uint32_t b, uint32_t accumulate) {
    const uint64_t adesc = make_desc(a), bdesc = make_desc(b);
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(kPollNs)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tma_reduce_add3(const CUtensorMap* map, int x, int y, int z, uint32_t src) {
    asm volatile(
        "cp.reduce.async.bulk.tensor.3d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(x), "r"(y), "r"(z), "r"(src)
        : "memory");
}

// 32 consecutive fp32 columns of this warp's 32 TMEM lanes (one register per column)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

// sum[c] += TMEM[lane][col + c] for the 128 columns at col (two 32-column loads per wait)
__device__ __forceinline__ void add_tmem_row(uint32_t col, float (&sum)[kTN]) {
#pragma unroll
    for (int j = 0; j < kTN / 32; j += 2) {
        uint32_t v[32], w[32];
        tmem_ld32(col + uint32_t(32 * j), v);
        tmem_ld32(col + uint32_t(32 * j + 32), w);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            sum[32 * j + i] += __uint_as_float(v[i]);
            sum[32 * j + 32 + i] += __uint_as_float(w[i]);
        }
    }
}

struct TcArgs {
    int cx0, cx1;     // real columns [2 c0, 2 c1) of C
    int cy0, cy1;     // rows [r0, r1) of C
    int nk;           // K slices of kTK elements
    uint32_t limit;   // spin limit of the pipeline waits
    int32_t* err;
    int kpd;          // K steps (of 16) accumulated in TMEM between two drains: 1, 2 or 4
    int tiles_x, tiles_y, ntiles;   // 128 x 128 tiles of C per matrix, and over the batch
    int bx0;          // first K element of the B planes (their rows may hold more of K)
};

// Persistent: CTA c takes tiles c, c + gridDim.x, ... (x fastest, then y, then the batch member);
// the slice counter g and the drain-unit counter u run on across tiles, so the loads and MMAs of
// the next tile overlap the last drains and the output of the previous one.
// barrier slots: full[S], empty[S], accf[2] (big buffer written), acce[2] (big buffer drained), done,
// smle[2] (small buffer of a tile drained)
template <int NP>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, TcArgs a) {
    constexpr int S = Cfg<NP>::kStages;
    constexpr int SB = Cfg<NP>::kStageBytes;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char* ops = smem_raw + pad;
    const uint32_t ops_s = raw + pad;
    const uint32_t stage_out = ops_s + uint32_t(S) * SB;   // 4 drain warps x 2 x 4 KiB of output staging
    uint64_t* bars = reinterpret_cast<uint64_t*>(ops + size_t(S) * SB + kStagingBytes);
    constexpr int kBars = 2 * S + 7;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kBars);
    volatile int* s_abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* s_issued = s_abort + 1;
    volatile int* s_consumed = s_abort + 2;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[S]), accf0 = smem_u32(&bars[2 * S]),
                   acce0 = smem_u32(&bars[2 * S + 2]), done = smem_u32(&bars[2 * S + 4]),
                   smle0 = smem_u32(&bars[2 * S + 5]);
    const int per_tile = a.tiles_x * a.tiles_y;
    const int upb = (kTK / 16) / a.kpd;   // drain units per slice

    if (tid == 0) {
        *s_abort = 0;
        *s_issued = 0;
        *s_consumed = 0;
        for (int i = 0; i < kBars; ++i) {
            // acce and smle: one arrive per drain warp
            const uint32_t cnt = ((i >= 2 * S + 2 && i < 2 * S + 4) || i >= 2 * S + 5) ? 4u : 1u;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[i])), "r"(cnt));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmC)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    if (tid == 0) {
        // TMA producer: NP planes of A, then NP planes of B, per slice
        int g = 0;
        bool stop = false;
        for (int t = blockIdx.x; t < a.ntiles && !stop; t += gridDim.x) {
            const int f = t / per_tile, rem = t - f * per_tile, by = rem / a.tiles_x, bx = rem - by * a.tiles_x;
            for (int kt = 0; kt < a.nk; ++kt, ++g) {
                const int s = g % S;
                if (g >= S && !mbar_wait(empty0 + 8u * s, uint32_t((g / S - 1) & 1), a.limit)) {
                    *s_abort = 1;
                    stop = true;
                    break;
                }
                if (*s_abort) {
                    stop = true;
                    break;
                }
                const uint32_t base = ops_s + uint32_t(s) * SB;
                const uint32_t fb = full0 + 8u * s;
                expect_tx(fb, SB);
                const int x = kt * kTK;
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    tma_load3(base + q * kPlaneBytes, &tmA, x, by * kTM, NP * f + q, fb);
                    tma_load3(base + (NP + q) * kPlaneBytes, &tmB, a.bx0 + x, bx * kTN, NP * f + q, fb);
                }
            }
        }
        *s_issued = g;
    } else if (tid == 32) {
        // MMA issuer: drain unit u (a.kpd K steps of 16) accumulates its big products into TMEM
        // columns 128 (u & 1); the small products of the tile this CTA takes as its tl-th go to
        // columns 256 + 128 (tl & 1); the drain warps empty a buffer before it is used again
        int g = 0, u = 0, tl = 0;
        bool stop = false;
        for (int t = blockIdx.x; t < a.ntiles && !stop; t += gridDim.x, ++tl) {
            const uint32_t tsmall = tmem + 256u + uint32_t(tl & 1) * 128u;
            if (NP == 3 && tl >= 2 && !mbar_wait(smle0 + 8u * (tl & 1), uint32_t((tl / 2 - 1) & 1), a.limit)) {
                *s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            bool first = true;   // first K step of the tile: the small sums start from zero
            for (int kt = 0; kt < a.nk && !stop; ++kt) {
                const int s = g % S;
                if (!mbar_wait(full0 + 8u * s, uint32_t((g / S) & 1), a.limit)) {
                    *s_abort = 1;
                    stop = true;
                    break;
                }
                ++g;   // this stage's loads have landed
                if (*s_abort) {
                    stop = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t base = ops_s + uint32_t(s) * SB;
                for (int ui = 0; ui < upb; ++ui, ++u) {
                    const int b = u & 1;
                    if (u >= 2 && !mbar_wait(acce0 + 8u * b, uint32_t((u / 2 - 1) & 1), a.limit)) {
                        *s_abort = 1;
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t tbig = tmem + uint32_t(b) * 128u;
                    for (int kk = 0; kk < a.kpd; ++kk) {
                        const int ks = ui * a.kpd + kk;   // K = 16 per MMA: 32 bytes along the swizzle row
                        const uint32_t off = uint32_t(ks) * 32u;
                        const uint32_t acc = kk == 0 ? 0u : 1u, accs = first ? 0u : 1u;
                        first = false;
                        const uint32_t A0 = base + off, B0 = base + NP * kPlaneBytes + off;
                        mma_bf16(tbig, A0, B0, acc);
                        if constexpr (NP == 3) {
                            const uint32_t A1 = A0 + kPlaneBytes, A2 = A0 + 2 * kPlaneBytes;
                            const uint32_t B1 = B0 + kPlaneBytes, B2 = B0 + 2 * kPlaneBytes;
                            mma_bf16(tsmall, A0, B1, accs);
                            mma_bf16(tsmall, A1, B0, 1u);
                            mma_bf16(tsmall, A0, B2, 1u);
                            mma_bf16(tsmall, A2, B0, 1u);
                            mma_bf16(tsmall, A1, B1, 1u);
                        }
                    }
                    mma_commit(accf0 + 8u * b);
                }
                if (stop) break;
                mma_commit(empty0 + 8u * s);
            }
        }
        *s_consumed = g;
        mma_commit(done);   // tracks every MMA issued above
    } else if (warp >= 4) {
        // drain warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 = tile rows, all 128 columns
        const int q = warp & 3;
        const uint32_t trow = tmem + (uint32_t(32 * q) << 16);
        const uint32_t stage0 = stage_out + uint32_t(warp - 4) * 8192u;
        const int nu = a.nk * upb;   // drain units per tile
        int u = 0, outs = 0, tl = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++tl) {
            const int f = t / per_tile, rem = t - f * per_tile, by = rem / a.tiles_x, bx = rem - by * a.tiles_x;
            float sum[kTN];
#pragma unroll
            for (int j = 0; j < kTN; ++j) sum[j] = 0.f;
            for (int uu = 0; uu < nu; ++uu, ++u) {
                const int b = u & 1;
                if (!mbar_wait(accf0 + 8u * b, uint32_t((u / 2) & 1), a.limit)) {
                    ok = false;
                    *s_abort = 1;
                    break;
                }
                if (*s_abort) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                add_tmem_row(trow + uint32_t(b) * 128u, sum);
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(acce0 + 8u * b);
            }
            if (!ok) break;
            if constexpr (NP == 3) {
                // the tile's last commit covered every MMA of the tile, the small products included
                add_tmem_row(trow + 256u + uint32_t(tl & 1) * 128u, sum);
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) mbar_arrive(smle0 + 8u * (tl & 1));
            }
            // -sum into C through the dedicated staging buffers (alternating; a buffer is written
            // again only after the reduce two commits back has read it)
            const int y = a.cy0 + by * kTM + 32 * q;
            const int nch = y < a.cy1 ? min(kTN / 32, (a.cx1 - a.cx0 - bx * kTN + 31) / 32) : 0;
#pragma unroll
            for (int ch = 0; ch < kTN / 32; ++ch) {
                if (ch >= nch) break;
                const uint32_t stg = stage0 + uint32_t(outs & 1) * 4096u;
                if (outs >= 2) {
                    if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    __syncwarp();
                }
#pragma unroll
                for (int c4 = 0; c4 < 8; ++c4) {
                    const uint32_t addr = stg + uint32_t(lane) * 128u + (uint32_t(c4 ^ (lane & 7)) << 4);
                    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(-sum[32 * ch + 4 * c4]),
                                 "f"(-sum[32 * ch + 4 * c4 + 1]), "f"(-sum[32 * ch + 4 * c4 + 2]),
                                 "f"(-sum[32 * ch + 4 * c4 + 3])
                                 : "memory");
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    tma_reduce_add3(&tmC, a.cx0 + bx * kTN + ch * 32, y, f, stg);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
                __syncwarp();
                ++outs;
            }
        }
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }
    __syncthreads();
    // drain: loads and MMAs already issued finish before shared or tensor memory is released
    if (tid == 0) {
        bool ok = true;
        for (int g = *s_consumed; g < *s_issued; ++g)
            ok = mbar_wait(full0 + 8u * (g % S), uint32_t((g / S) & 1), kDrainSpin) && ok;
        if (!ok || *s_abort) atomicExch(a.err, 1);
    }
    if (tid == 32 && !mbar_wait(done, 0u, kDrainSpin)) atomicExch(a.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }
inline size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

int sm_count() {
    static int n = [] {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

// one persistent CTA per SM (the shared memory allows one), at most one per tile
template <int NP>
void launch_gemm_kernel(const CUtensorMap& mA, const CUtensorMap& mB, const CUtensorMap& mC, TcArgs args, int M,
                        int N, int F, cudaStream_t st) {
    args.tiles_x = int(cdiv(2 * int64_t(N), kTN));
    args.tiles_y = int(cdiv(M, kTM));
    args.ntiles = args.tiles_x * args.tiles_y * F;
    const int grid = std::min(args.ntiles, sm_count());
    tc_gemm_kernel<NP><<<grid, kThreads, Cfg<NP>::kSmem, st>>>(mA, mB, mC, args);
}

// 3-D tensor map: inner dimension d0 (contiguous), rows d1 (stride s1 bytes), planes d2 (stride s2).
bool encode3(CUtensorMap* map, CUtensorMapDataType dt, void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1,
             uint64_t s2, uint32_t box0, uint32_t box1, CUtensorMapL2promotion l2) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {s1, s2};
    const cuuint32_t box[3] = {box0, box1, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(map, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, l2,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// BF16 elements of the packed operands of one matrix: NP planes of rows x Kp
int64_t pack_elems(int np, int64_t rows, int64_t Kp) { return np * rows * Kp; }

template <int NP>
bool launch_np(float2* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1, int k0, int K, const TcCtx& tc,
               cudaStream_t st) {
    const int M = r1 - r0, N = c1 - c0;
    const int64_t Kp = round_up(2 * int64_t(K), kTK);
    const int64_t aE = int64_t(F) * pack_elems(NP, M, Kp), bE = int64_t(F) * pack_elems(NP, 2 * int64_t(N), Kp);
    const size_t need = size_t(aE + bE) * sizeof(__nv_bfloat16) + 256;
    if (!tc.ws || need > tc.ws_bytes) return false;
    auto* Ap = reinterpret_cast<__nv_bfloat16*>((reinterpret_cast<uintptr_t>(tc.ws) + 255) & ~uintptr_t(255));
    __nv_bfloat16* Bp = Ap + aE;   // aE is a multiple of 64 elements: Bp stays 128-byte aligned

    CUtensorMap mA, mB, mC;
    if (!encode3(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Ap, Kp, M, uint64_t(NP) * F, Kp * 2, uint64_t(M) * Kp * 2,
                 kTK, kTM, CU_TENSOR_MAP_L2_PROMOTION_L2_256B) ||
        !encode3(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Bp, Kp, 2 * uint64_t(N), uint64_t(NP) * F, Kp * 2,
                 2 * uint64_t(N) * Kp * 2, kTK, kTN, CU_TENSOR_MAP_L2_PROMOTION_L2_256B) ||
        !encode3(&mC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, G, 2 * uint64_t(c1), uint64_t(r1), uint64_t(F),
                 uint64_t(ld) * 8, uint64_t(sG) * 8, 32, 32, CU_TENSOR_MAP_L2_PROMOTION_NONE))
        return false;

    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(tc_gemm_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg<NP>::kSmem));
        attr_set = true;
    }
    {
        ProfScope ps(PK_PACK, 0.0, st);
        pack_a_kernel<NP><<<dim3(cdiv(int64_t(M) * Kp / 8, 256), F), 256, 0, st>>>(
            reinterpret_cast<const float*>(G), 2 * sG, 2 * int64_t(ld), r0, M, 2 * k0, 2 * K, int(Kp), Ap);
        pack_b_kernel<NP><<<dim3(cdiv(Kp / 2, 32), cdiv(N, 32), F), dim3(32, 8), 0, st>>>(G, sG, ld, k0, K, c0, N,
                                                                                          int(Kp), 0, int(Kp / 2), Bp);
    }
    TcArgs args{2 * c0, 2 * c1, r0, r1, int(Kp / kTK), g_spin_limit.load(), tc.err, drain_ksteps(), 0, 0, 0, 0};
    ProfScope ps(PK_TCGEMM, 8.0 * F * double(M) * double(N) * K, st);
    launch_gemm_kernel<NP>(mA, mB, mC, args, M, N, F, st);
    return true;
}

// The U12 columns of a slab step, packed once: rows of U12 are final after their block's triangle
// solve, so each block is packed when it is done and every later update (the left-looking solve
// of the blocks below, the Schur update) reads the same planes.  A is packed per update.
template <int NP>
bool launch_np_lazy(float2* G, int64_t sG, int ld, int F, int r0, int r1, int k0, int K, const TcCtx& tc,
                    cudaStream_t st) {
    const int M = r1 - r0, N = tc.bN, c0 = tc.bc0, c1 = tc.bc0 + tc.bN;
    const int64_t Kp = round_up(2 * int64_t(K), kTK);
    const int64_t aE = int64_t(F) * pack_elems(NP, M, Kp);
    // the packed rows start at K element 2 k0, which the slices must meet on their 64-element grid
    if ((2 * k0) % kTK || 2 * k0 + Kp > tc.bKp || size_t(aE) * sizeof(__nv_bfloat16) + 256 > tc.a_bytes)
        return false;
    auto* Ap = reinterpret_cast<__nv_bfloat16*>((reinterpret_cast<uintptr_t>(tc.ws) + 255) & ~uintptr_t(255));
    auto* Bp = static_cast<__nv_bfloat16*>(tc.bpack);
    CUtensorMap mA, mB, mC;
    if (!encode3(&mA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Ap, Kp, M, uint64_t(NP) * F, Kp * 2, uint64_t(M) * Kp * 2,
                 kTK, kTM, CU_TENSOR_MAP_L2_PROMOTION_L2_256B) ||
        !encode3(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, Bp, tc.bKp, 2 * uint64_t(N), uint64_t(NP) * F, tc.bKp * 2,
                 2 * uint64_t(N) * tc.bKp * 2, kTK, kTN, CU_TENSOR_MAP_L2_PROMOTION_L2_256B) ||
        !encode3(&mC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, G, 2 * uint64_t(c1), uint64_t(r1), uint64_t(F),
                 uint64_t(ld) * 8, uint64_t(sG) * 8, 32, 32, CU_TENSOR_MAP_L2_PROMOTION_NONE))
        return false;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(tc_gemm_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(Cfg<NP>::kSmem));
        attr_set = true;
    }
    {
        ProfScope ps(PK_PACK, 0.0, st);
        pack_a_kernel<NP><<<dim3(cdiv(int64_t(M) * Kp / 8, 256), F), 256, 0, st>>>(
            reinterpret_cast<const float*>(G), 2 * sG, 2 * int64_t(ld), r0, M, 2 * k0, 2 * K, int(Kp), Ap);
    }
    TcArgs args{2 * c0, 2 * c1, r0, r1, int(Kp / kTK), g_spin_limit.load(), tc.err, drain_ksteps(), 0, 0, 0,
                2 * k0};
    ProfScope ps(PK_TCGEMM, 8.0 * F * double(M) * double(N) * K, st);
    launch_gemm_kernel<NP>(mA, mB, mC, args, M, N, F, st);
    return true;
}

}  // namespace

void set_tc_spin_limit(uint32_t spins) { g_spin_limit.store(spins ? spins : kDefaultSpin); }

size_t tc_workspace_bytes(int F, int m, int ncols, int npiv, int planes) {
    const int64_t nb = std::min(128, npiv);
    const int64_t Kpn = round_up(2 * int64_t(npiv), kTK), Kp1 = round_up(2 * nb, kTK);
    int64_t a = pack_elems(planes, m - nb, Kp1);
    a = std::max(a, pack_elems(planes, std::min(128, npiv), Kpn));
    a = std::max(a, pack_elems(planes, m - npiv, Kpn));
    int64_t b = pack_elems(planes, 2 * (npiv - nb), Kp1);
    b = std::max(b, pack_elems(planes, 2 * int64_t(ncols - npiv), Kpn));
    return size_t(F) * size_t(a + b) * sizeof(__nv_bfloat16) + 1024;
}

bool launch_tc_update(float2* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1, int k0, int K,
                      const TcCtx& tc, cudaStream_t st) {
    if (r1 <= r0 || c1 <= c0 || K <= 0) return true;
    // TMA: 16-byte aligned base and row / matrix strides, tile columns start on 16-byte boundaries
    if ((reinterpret_cast<uintptr_t>(G) & 15) || (ld & 1) || (sG & 1) || (c0 & 1)) return false;
    return tc.planes == 1 ? launch_np<1>(G, sG, ld, F, r0, r1, c0, c1, k0, K, tc, st)
                          : launch_np<3>(G, sG, ld, F, r0, r1, c0, c1, k0, K, tc, st);
}

size_t tc_a_region_bytes(int F, int m, int ncols, int npiv, int planes) {
    const int64_t nb = std::min(128, npiv);
    const int64_t Kpn = round_up(2 * int64_t(npiv), kTK), Kp1 = round_up(2 * nb, kTK);
    int64_t a = pack_elems(planes, m - nb, Kp1);
    a = std::max(a, pack_elems(planes, std::min(128, npiv), Kpn));
    a = std::max(a, pack_elems(planes, m - npiv, Kpn));
    return align_up(size_t(F) * size_t(a) * sizeof(__nv_bfloat16) + 256);
}

bool tc_begin_lazy(float2* G, int64_t sG, int ld, int F, int npiv, int c0, int c1, TcCtx& tc, cudaStream_t st) {
    tc.bpack = nullptr;
    if ((reinterpret_cast<uintptr_t>(G) & 15) || (ld & 1) || (sG & 1) || (c0 & 1) || c1 <= c0 || !tc.ws) return false;
    const int64_t Kp = round_up(2 * int64_t(npiv), kTK);
    const size_t bytes = size_t(F) * size_t(pack_elems(tc.planes, 2 * int64_t(c1 - c0), Kp)) * sizeof(__nv_bfloat16);
    if (tc.a_bytes + bytes > tc.ws_bytes) return false;
    tc.bpack = static_cast<char*>(tc.ws) + tc.a_bytes;   // a_bytes is a multiple of 256
    tc.bKp = Kp;
    tc.bN = c1 - c0;
    tc.bc0 = c0;
    // the K padding beyond 2 npiv must read as zero
    return cudaMemsetAsync(tc.bpack, 0, bytes, st) == cudaSuccess;
}

void tc_pack_b_rows(float2* G, int64_t sG, int ld, int F, int k_begin, int k_end, const TcCtx& tc, cudaStream_t st) {
    if (!tc.bpack || k_end <= k_begin) return;
    const int K = k_end - k_begin;
    ProfScope ps(PK_PACK, 0.0, st);
    auto* Bp = static_cast<__nv_bfloat16*>(tc.bpack);
    const dim3 grid(cdiv(K, 32), cdiv(tc.bN, 32), F);
    if (tc.planes == 1)
        pack_b_kernel<1><<<grid, dim3(32, 8), 0, st>>>(G, sG, ld, k_begin, K, tc.bc0, tc.bN, int(tc.bKp), 2 * k_begin,
                                                        K, Bp);
    else
        pack_b_kernel<3><<<grid, dim3(32, 8), 0, st>>>(G, sG, ld, k_begin, K, tc.bc0, tc.bN, int(tc.bKp), 2 * k_begin,
                                                        K, Bp);
}

bool launch_tc_update_lazy(float2* G, int64_t sG, int ld, int F, int r0, int r1, int k0, int K, const TcCtx& tc,
                           cudaStream_t st) {
    if (!tc.bpack) return false;
    if (r1 <= r0 || K <= 0) return true;
    return tc.planes == 1 ? launch_np_lazy<1>(G, sG, ld, F, r0, r1, k0, K, tc, st)
                          : launch_np_lazy<3>(G, sG, ld, F, r0, r1, k0, K, tc, st);
}

}  // namespace fsi

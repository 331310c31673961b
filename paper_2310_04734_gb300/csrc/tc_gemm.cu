// Trailing update of the band LU on the 5th-generation tensor cores (tcgen05).
//
//   C[r0:r1, c0:c1] -= A[r0:r1, k0:k0+K] * B[k0:k0+K, c0:c1]      (complex FP32, row major)
//
// The complex product is one real GEMM on interleaved storage: with A' the
// M x 2K real view of A and B' the 2K x 2N real matrix with 2x2 blocks
// [[Br, Bi], [-Bi, Br]], C' -= A' B' is exactly the complex update on the
// interleaved C.  FP32 accuracy is kept on the TF32 tensor pipe by splitting
// every operand into hi = tf32(x) and lo = tf32(x - hi) and accumulating
// hi*hi + hi*lo + lo*hi in FP32.  Plain TF32 products are not accurate enough
// for the refinement of these systems to converge.  hi*hi and the two cross
// terms accumulate in separate TMEM accumulators, added in FP32 only in the
// epilogue: the tensor core aligns products to the accumulator's exponent and
// truncates, which would drop most of the small cross terms if they were added
// into the large hi*hi sum.
//
// One CTA (8 warps) per 128 x 256 real tile.  For each 32-float K slice the
// threads load A' and B' from global memory (vector loads), split them and
// store whole 16-byte chunks into shared memory in the 128-byte-swizzled
// K-major layout the MMA descriptors describe; two slice buffers alternate and
// the next slice is prefetched into registers while the current slice's MMAs
// run.  One thread issues tcgen05.mma (M=128, N=256, K=8, kind::tf32) and
// commits to an mbarrier per buffer.  The epilogue reads both accumulators with
// tcgen05.ld, stages them through shared memory and subtracts them from C with
// coalesced row accesses.  Every mbarrier wait is bounded: on timeout the CTA
// records an error, stops issuing work, and still frees its tensor memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.cuh"
#include "prof.h"

namespace fsi {

namespace {

constexpr int kTM = 128;            // real rows per tile (MMA M)
constexpr int kTN = 256;            // real columns per tile (MMA N)
constexpr int kTK = 32;             // real K per shared-memory slice (one 128-byte swizzle row)
constexpr int kThreads = 256;
constexpr int kTmemCols = 512;      // two 256-column fp32 accumulators: hi*hi, and hi*lo + lo*hi
constexpr uint32_t kSpinLimit = 1u << 26;

// shared memory: per stage A_hi, A_lo (kTM x 128 B), B_hi, B_lo (kTN x 128 B)
constexpr int kABytes = kTM * 128;
constexpr int kBBytes = kTN * 128;
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;   // 96 KiB
constexpr int kStages = 2;
constexpr size_t kSmemBytes = size_t(kStages) * kStageBytes + 1024 + 64;

// per-thread items of one slice: A' 128 rows x 8 chunks, B 128 complex columns x 8 chunks
constexpr int kAItems = (kTM * (kTK / 4)) / kThreads;            // 4
constexpr int kBItems = ((kTN / 2) * (kTK / 4)) / kThreads;      // 4

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of the 16-byte chunk c (k = 4c..4c+3) of row `row` of a K-major tile with
// 128-byte rows in the 128-byte swizzle: chunk index XOR (row mod 8), 8-row groups of 1024 B
__device__ __forceinline__ uint32_t sw128_chunk(int row, int c) {
    return uint32_t(row) * 128u + (uint32_t(c ^ (row & 7)) << 4);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// hi / lo split of four values written as two 16-byte chunks
__device__ __forceinline__ void put_split(uint32_t hi_addr, uint32_t lo_addr, float4 v) {
    const float h0 = to_tf32(v.x), h1 = to_tf32(v.y), h2 = to_tf32(v.z), h3 = to_tf32(v.w);
    st_shared_v4(hi_addr, h0, h1, h2, h3);
    st_shared_v4(lo_addr, to_tf32(v.x - h0), to_tf32(v.y - h1), to_tf32(v.z - h2), to_tf32(v.w - h3));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFFu) >> 4);          // start address
    d |= uint64_t(1024u >> 4) << 32;                // stride byte offset
    d |= uint64_t(1) << 46;                         // descriptor version
    d |= uint64_t(2) << 61;                         // 128-byte swizzle
    return d;
}

// instruction descriptor: D f32, A/B tf32, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(kTN >> 3) << 17) | (uint32_t(kTM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (uint32_t it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
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

struct SliceRegs {
    float4 a[kAItems];
    float2 b0[kBItems], b1[kBItems];
};

__global__ void __launch_bounds__(kThreads, 1) tc_update_kernel(float2* G, int64_t sG, int ld, int r0, int r1, int c0,
                                                                int c1, int k0, int K, int32_t* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char* ops = smem_raw + pad;
    const uint32_t ops_s = raw + pad;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(ops + size_t(kStages) * kStageBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + kStages);
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int f = blockIdx.z;
    const float2* Gc = G + f * sG;
    float* Gf = reinterpret_cast<float*>(G + f * sG);
    const int64_t ldf = 2 * int64_t(ld);           // floats per row
    const int rt = r0 + blockIdx.y * kTM;          // first C row of the tile
    const int nt = c0 + blockIdx.x * (kTN / 2);    // first complex C column of the tile
    const int Kr = 2 * K;                          // real K

    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < kStages; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    // global -> registers for slice sl
    auto load_slice = [&](int sl, SliceRegs& R) {
        const int kb = sl * kTK;
#pragma unroll
        for (int it = 0; it < kAItems; ++it) {
            const int idx = tid + it * kThreads;
            const int r = idx >> 3, c = idx & 7;           // row, 16-byte chunk
            const int gr = rt + r, gk = kb + 4 * c;        // real k of the chunk's first float
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gr < r1) {
                const float* src = Gf + int64_t(gr) * ldf + 2 * k0 + gk;
                if (gk + 3 < Kr && (reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
                    v = *reinterpret_cast<const float4*>(src);   // only when the address is 16-byte aligned
                } else {
                    if (gk + 0 < Kr) v.x = src[0];
                    if (gk + 1 < Kr) v.y = src[1];
                    if (gk + 2 < Kr) v.z = src[2];
                    if (gk + 3 < Kr) v.w = src[3];
                }
            }
            R.a[it] = v;
        }
#pragma unroll
        for (int it = 0; it < kBItems; ++it) {
            const int idx = tid + it * kThreads;
            const int c = idx >> 7, nn = idx & 127;        // chunk c covers complex k 2c, 2c+1 of the slice
            const int n = nt + nn;
            const int j = (kb >> 1) + 2 * c;               // complex k within the panel
            float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
            if (n < c1) {
                if (j < K) v0 = Gc[int64_t(k0 + j) * ld + n];
                if (j + 1 < K) v1 = Gc[int64_t(k0 + j + 1) * ld + n];
            }
            R.b0[it] = v0;
            R.b1[it] = v1;
        }
    };
    // registers -> split, swizzled shared memory of stage st
    auto store_slice = [&](int st, const SliceRegs& R) {
        const uint32_t base = ops_s + uint32_t(st) * kStageBytes;
        const uint32_t Ahi = base, Alo = base + kABytes, Bhi = base + 2 * kABytes, Blo = base + 2 * kABytes + kBBytes;
#pragma unroll
        for (int it = 0; it < kAItems; ++it) {
            const int idx = tid + it * kThreads;
            const int r = idx >> 3, c = idx & 7;
            const uint32_t o = sw128_chunk(r, c);
            put_split(Ahi + o, Alo + o, R.a[it]);
        }
#pragma unroll
        for (int it = 0; it < kBItems; ++it) {
            const int idx = tid + it * kThreads;
            const int c = idx >> 7, nn = idx & 127;
            const float2 p = R.b0[it], q = R.b1[it];
            // row 2n: (Br, -Bi) per complex k; row 2n+1: (Bi, Br)
            const uint32_t o0 = sw128_chunk(2 * nn, c), o1 = sw128_chunk(2 * nn + 1, c);
            put_split(Bhi + o0, Blo + o0, make_float4(p.x, -p.y, q.x, -q.y));
            put_split(Bhi + o1, Blo + o1, make_float4(p.y, p.x, q.y, q.x));
        }
    };

    const int nslices = (Kr + kTK - 1) / kTK;
    uint32_t phase[kStages] = {0, 0};
    SliceRegs regs;
    load_slice(0, regs);
    for (int sl = 0; sl < nslices; ++sl) {
        const int st = sl % kStages;
        if (sl >= kStages) {   // the MMAs that read this buffer must be done
            if (!mbar_wait(smem_u32(&mbar[st]), phase[st])) {
                if (tid == 0) { s_abort = 1; atomicExch(err, 1); }
            }
            phase[st] ^= 1u;
        }
        __syncthreads();
        if (s_abort) break;
        store_slice(st, regs);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t base = ops_s + uint32_t(st) * kStageBytes;
            const uint32_t ahi = base, alo = base + kABytes, bhi = base + 2 * kABytes, blo = base + 2 * kABytes + kBBytes;
#pragma unroll
            for (int s = 0; s < kTK / 8; ++s) {   // K = 8 per MMA: 32 bytes along the swizzle row
                const uint32_t off = uint32_t(s) * 32u;
                const uint32_t first = (sl == 0 && s == 0) ? 0u : 1u;
                mma_tf32(tmem, make_desc(ahi + off), make_desc(bhi + off), first);
                mma_tf32(tmem + 256u, make_desc(ahi + off), make_desc(blo + off), first);
                mma_tf32(tmem + 256u, make_desc(alo + off), make_desc(bhi + off), 1u);
            }
            mma_commit(smem_u32(&mbar[st]));
        }
        if (sl + 1 < nslices) load_slice(sl + 1, regs);   // overlaps the MMAs just issued
    }
    // the last commit tracks every MMA issued before it
    if (!s_abort) {
        const int st = (nslices - 1) % kStages;
        if (!mbar_wait(smem_u32(&mbar[st]), phase[st])) {
            if (tid == 0) atomicExch(err, 1);
            s_abort = 1;
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    if (!s_abort) {
        // warp w: TMEM lanes 32*(w%4).., column half w/4; staged through its own 32 x 33 tile
        float* tile = reinterpret_cast<float*>(ops) + warp * (32 * 33);
        const int lane_base = (warp & 3) * 32;
        const int half = warp >> 2;
        for (int cb = half * 128; cb < half * 128 + 128; cb += 32) {
            uint32_t v[32], u[32];
            const uint32_t taddr = tmem + (uint32_t(lane_base) << 16) + uint32_t(cb);
            tmem_ld32(taddr, v);
            tmem_ld32(taddr + 256u, u);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(v[j]) + __uint_as_float(u[j]);
            __syncwarp();
            const int q = 2 * nt + cb + lane;             // real column of C handled by this lane
            const bool qok = q < 2 * c1;
            for (int rr = 0; rr < 32; ++rr) {
                const int row = rt + lane_base + rr;
                if (row < r1 && qok) Gf[int64_t(row) * ldf + q] -= tile[rr * 33 + lane];
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

inline unsigned cdiv(int64_t a, int64_t b) { return unsigned((a + b - 1) / b); }

}  // namespace

void launch_tc_update(float2* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1, int k0, int K,
                      int32_t* err, cudaStream_t st) {
    if (r1 <= r0 || c1 <= c0 || K <= 0) return;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(tc_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemBytes));
        attr_set = true;
    }
    dim3 grid(cdiv(int64_t(c1 - c0), kTN / 2), cdiv(r1 - r0, kTM), F);
    ProfScope ps(PK_GEMM, 8.0 * F * double(r1 - r0) * double(c1 - c0) * K, st);
    tc_update_kernel<<<grid, kThreads, kSmemBytes, st>>>(G, sG, ld, r0, r1, c0, c1, k0, K, err);
}

}  // namespace fsi

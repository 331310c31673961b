// Complex FP32 update C[r0:r1, c0:c1] -= A[r0:r1, k0:k0+K] * B[k0:k0+K, c0:c1]
// inside each matrix of a batch (row major, all three blocks in the same matrix):
// the trailing update of the band LU's right-looking partial factorisation, and
// the updates inside its outer panels.
//
// SIMT kernel on the FP32 FMA pipe.  One CTA of 256 threads computes a
// 128 x 64 complex tile; each thread owns 8 x 4 complex accumulators (rows
// 4*ty..4*ty+3 and 64+4*ty.., columns 2*tx, 2*tx+1 and 32+2*tx, 33+2*tx), so one
// K step costs six 16-byte shared loads for 128 FMAs.  K is staged 16 at a time
// in two shared-memory buffers: the next slice is copied from global memory by
// cp.async (no staging registers) while the current one is multiplied.  Two
// CTAs fit per SM, so one CTA's epilogue (the read-modify-write of C, whose
// lines are prefetched into L2 when the CTA starts) overlaps the other's FMAs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"
#include "prof.h"

namespace fsi {

namespace {

constexpr int kCM = 128, kCN = 64, kCK = 16, kCT = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 8-byte asynchronous global -> shared copy; writes zeros when !ok (no bytes read)
__device__ __forceinline__ void cp_async8(uint32_t saddr, const void* g, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(saddr), "l"(g), "r"(ok ? 8 : 0) : "memory");
}

__global__ void __launch_bounds__(kCT, 2) cgemm_f32_kernel(float2* __restrict__ G, int64_t sG, int ld, int r0, int r1,
                                                           int c0, int c1, int k0, int K, bool vec_ok) {
    __shared__ __align__(16) float2 As[2][kCK][kCM];
    __shared__ __align__(16) float2 Bs[2][kCK][kCN];
    const int f = blockIdx.z;
    float2* A = G + f * sG;
    const int rb = r0 + blockIdx.y * kCM, cb = c0 + blockIdx.x * kCN;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const float2 z = make_float2(0.f, 0.f);

    // global -> shared copies (cp.async, zero-filled outside the block):
    // A row la_r, k in [la_k, la_k+8) stored transposed; B k row lb_k, columns [lb_c, lb_c+4)
    const int la_r = tid & (kCM - 1), la_k = (tid >> 7) * 8;   // a warp fills 32 consecutive rows of As
    const int lb_k = tid >> 4, lb_c = (tid & 15) * 4;
    const bool a_ok = rb + la_r < r1;
    const float2* a_src = A + int64_t(min(rb + la_r, r1 - 1)) * ld + k0 + la_k;
    auto issue = [&](int kb, int s) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const bool ok = a_ok && kb + la_k + q < K;
            cp_async8(smem_u32(&As[s][la_k + q][la_r]), ok ? a_src + kb + q : A, ok);
        }
        const int gk = kb + lb_k;
        const float2* b_src = A + int64_t(k0 + min(gk, K - 1)) * ld + cb + lb_c;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool ok = gk < K && cb + lb_c + q < c1;
            cp_async8(smem_u32(&Bs[s][lb_k][lb_c + q]), ok ? b_src + q : A, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    // the C tile is read-modify-written at the end: start pulling it into L2 now
    {
        const int pr = tid >> 1;
        if (rb + pr < r1) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = cb + ((tid & 1) * 2 + h) * 16;   // 16 complex = one 128-byte line
                if (col < c1)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(A + int64_t(rb + pr) * ld + col));
            }
        }
    }

    float2 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = z;

    const int nk = (K + kCK - 1) / kCK;
    issue(0, 0);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int t = 0; t < nk; ++t) {
        const int s = t & 1;
        if (t + 1 < nk) issue((t + 1) * kCK, s ^ 1);
#pragma unroll
        for (int kk = 0; kk < kCK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[s][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[s][kk][ty * 4 + 2]);
            const float4 a2 = *reinterpret_cast<const float4*>(&As[s][kk][64 + ty * 4]);
            const float4 a3 = *reinterpret_cast<const float4*>(&As[s][kk][64 + ty * 4 + 2]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[s][kk][tx * 2]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[s][kk][32 + tx * 2]);
            const float2 a[8] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(a1.x, a1.y),
                                 make_float2(a1.z, a1.w), make_float2(a2.x, a2.y), make_float2(a2.z, a2.w),
                                 make_float2(a3.x, a3.y), make_float2(a3.z, a3.w)};
            const float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                                 make_float2(b1.z, b1.w)};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
    }
    // epilogue: columns 2*tx, 2*tx+1 (and 32 + those) are adjacent, so pairs move as 16 bytes
    const bool pairs = vec_ok && cb + kCN <= c1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int row = rb + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (row >= r1) continue;
        float2* crow = A + int64_t(row) * ld + cb;
        if (pairs) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float4* p = reinterpret_cast<float4*>(crow + h * 32 + tx * 2);
                float4 c = *p;
                c.x -= acc[i][2 * h].x;
                c.y -= acc[i][2 * h].y;
                c.z -= acc[i][2 * h + 1].x;
                c.w -= acc[i][2 * h + 1].y;
                *p = c;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int col = cb + (j < 2 ? tx * 2 + j : 32 + tx * 2 + (j - 2));
                if (col >= c1) continue;
                float2& c = A[int64_t(row) * ld + col];
                c = csub(c, acc[i][j]);
            }
        }
    }
}

}  // namespace

void launch_cgemm_f32(float2* G, int64_t sG, int ld, int F, int r0, int r1, int c0, int c1, int k0, int K,
                      cudaStream_t st) {
    if (r1 <= r0 || c1 <= c0 || K <= 0) return;
    dim3 grid(unsigned((c1 - c0 + kCN - 1) / kCN), unsigned((r1 - r0 + kCM - 1) / kCM), unsigned(F));
    ProfScope ps(PK_GEMM, 8.0 * F * double(r1 - r0) * double(c1 - c0) * K, st);
    // 16-byte epilogue access needs every tile's first column and every row start 16-byte aligned
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(G) & 15) == 0) && (ld % 2 == 0) && (c0 % 2 == 0) &&
                        (sG % 2 == 0);
    cgemm_f32_kernel<<<grid, kCT, 0, st>>>(G, sG, ld, r0, r1, c0, c1, k0, K, vec_ok);
}

}  // namespace fsi

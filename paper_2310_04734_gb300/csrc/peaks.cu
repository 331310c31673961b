// Throughput probes for the roofline denominators of this library's kernels:
// the FP32 and FP64 FMA pipes (SIMT) and the tcgen05 tensor pipe for BF16 and
// TF32 operands.  Each probe keeps one unit busy with independent operations
// and no memory traffic; the host times it with CUDA events on the caller's
// stream.  The values are those of the GPU at the clocks it runs at during the
// probe, so they are measured, not derived from unit counts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "fsi_internal.h"

namespace fsi {

namespace {

constexpr int kChains = 8;          // independent FMA chains per thread
constexpr int kUnroll = 16;
constexpr uint32_t kSpin = 1u << 26;

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T seed, T mul, int64_t iters, T* sink) {
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = seed + T(threadIdx.x + c);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], mul, seed);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == T(-12345.678)) sink[threadIdx.x] = s;   // keeps the chains live
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFFu) >> 4);
    d |= uint64_t(1024u >> 4) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(2) << 61;
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < kSpin; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One CTA per SM: M = 128, N = NN MMAs back to back on shared-memory operands (contents
// irrelevant), accumulating into TMEM; every 64 MMAs a commit and a wait bound the queue.
// KIND 0: kind::f16 with BF16 operands (K = 16 per MMA); 1: kind::tf32 (K = 8).  NN = 128 is the
// tile of the band LU's update kernel; NN = 256 is the widest single-CTA shape.
template <int KIND, int NN>
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int64_t groups, int32_t* err) {
    __shared__ __align__(1024) unsigned char ops[256 * 128];   // A: first 128 rows, B: all 256
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < int(sizeof(ops)) / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(ops)[i] = 0x3c003c00u;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tslot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tslot;
    if (tid == 0) {
        const uint64_t ad = make_desc(smem_u32(ops)), bd = make_desc(smem_u32(ops));
        constexpr uint32_t fmt = KIND == 0 ? 1u : 2u;   // BF16 (kind::f16) or TF32
        constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | (uint32_t(NN >> 3) << 17) |
                                   (uint32_t(128 >> 4) << 24);
        uint32_t phase = 0;
        for (int64_t g = 0; g < groups; ++g) {
#pragma unroll 8
            for (int i = 0; i < 64; ++i) {
                const uint32_t acc = (g == 0 && i == 0) ? 0u : 1u;
                if constexpr (KIND == 0)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                else
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar))
                         : "memory");
            if (!mbar_wait(smem_u32(&bar), phase)) {
                atomicExch(err, 1);
                // the MMAs already issued still complete before TMEM is freed below
                mbar_wait(smem_u32(&bar), phase);
                break;
            }
            phase ^= 1u;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace

}  // namespace fsi

using namespace fsi;

extern "C" fsi_status fsi_probe_peak(int kind, double seconds_hint, void* scratch, double* tflops_out,
                                     double* ms_out, void* stream) {
    if (!(tflops_out && scratch && kind >= 0 && kind <= 4)) {
        set_error("fsi_probe_peak: bad arguments");
        return FSI_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || sms <= 0) {
        set_error(std::string("fsi_probe_peak: ") + cudaGetErrorString(e));
        return FSI_ECUDA;
    }
    cudaMemsetAsync(scratch, 0, 1024, st);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const double hint = seconds_hint > 0 ? seconds_hint : 0.2;
    double flops_per_unit = 0.0;
    auto launch = [&](int64_t units) {
        switch (kind) {
            case 0:
                fma_probe_kernel<float><<<sms * 8, 256, 0, st>>>(1.0001f, 0.9999f, units,
                                                                static_cast<float*>(scratch));
                break;
            case 1:
                fma_probe_kernel<double><<<sms * 8, 256, 0, st>>>(1.0001, 0.9999, units,
                                                                 static_cast<double*>(scratch));
                break;
            case 2:
                mma_probe_kernel<0, 256><<<sms, 128, 0, st>>>(units, static_cast<int32_t*>(scratch));
                break;
            case 3:
                mma_probe_kernel<1, 256><<<sms, 128, 0, st>>>(units, static_cast<int32_t*>(scratch));
                break;
            default:
                mma_probe_kernel<0, 128><<<sms, 128, 0, st>>>(units, static_cast<int32_t*>(scratch));
                break;
        }
    };
    if (kind <= 1) flops_per_unit = 2.0 * kChains * kUnroll * 256.0 * sms * 8;
    else flops_per_unit = 64.0 * 2.0 * 128.0 * (kind == 4 ? 128.0 : 256.0) * (kind == 3 ? 8.0 : 16.0) * sms;
    // calibrate: grow the work until one launch takes about `hint` seconds
    int64_t units = kind <= 1 ? 256 : 16;
    float ms = 0.f;
    for (int rep = 0; rep < 12; ++rep) {
        cudaEventRecord(a, st);
        launch(units);
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) break;
        cudaEventElapsedTime(&ms, a, b);
        if (ms >= 1000.0 * hint * 0.5) break;
        units *= ms > 0.5f ? std::max<int64_t>(2, int64_t(1000.0 * hint / ms)) : 8;
    }
    // the timed launch
    if (e == cudaSuccess) {
        cudaEventRecord(a, st);
        launch(units);
        cudaEventRecord(b, st);
        e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    }
    int32_t err = 0;
    if (e == cudaSuccess && kind >= 2) e = cudaMemcpy(&err, scratch, sizeof(err), cudaMemcpyDeviceToHost);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) {
        set_error(std::string("fsi_probe_peak: ") + cudaGetErrorString(e));
        return FSI_ECUDA;
    }
    if (err) {
        set_error("fsi_probe_peak: a bounded wait of the MMA probe gave up");
        return FSI_ETIMEOUT;
    }
    *tflops_out = flops_per_unit * double(units) / (double(ms) * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return FSI_OK;
}

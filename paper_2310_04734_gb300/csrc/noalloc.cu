// Batched partial LU for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// running inside a memory pool or allocator that forbids new device
// allocations, real-time loops that must not block on the allocator, and
// hosts that embed the library behind an interface with no room for a scratch
// buffer.  fsi_batched_lu_noalloc serves them.  It runs the same kernels as
// fsi_batched_lu; the only scratch those kernels need -- one status flag per
// matrix (set when a pivot is zero or not finite), plus one counter -- lives
// in a fixed device array compiled into this library.  Every GPU that loads
// the library holds that array (16 KiB) until the process exits.
#include <cuda_runtime.h>

#include <sstream>
#include <string>

#include "fsi_internal.h"
#include "kernels.cuh"

namespace fsi {

namespace {

constexpr int kNoAllocMaxBatch = 4095;   // matrices per call; one more slot holds the counter

// Status flags [0, batch) and the singular-matrix counter [kNoAllocMaxBatch].
static __device__ __align__(256) int32_t g_lu_scratch[kNoAllocMaxBatch + 1];

__global__ void count_flags_kernel(const int32_t* flags, int batch, int32_t* counter) {
    int c = 0;
    for (int i = threadIdx.x; i < batch; i += blockDim.x) c += flags[i] != 0;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(counter, c);
}

// Device address of g_lu_scratch for the current device.  Looked up on every call: the lookup
// is host-side and cheap, and a cached address would dangle after the context is torn down and
// recreated (the module, and with it the array, may then load elsewhere).
fsi_status scratch_for_current_device(int32_t** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_lu_scratch);
    if (e != cudaSuccess || !p) {
        set_error(std::string("cudaGetSymbolAddress(g_lu_scratch): ") + cudaGetErrorString(e));
        return FSI_ECUDA;
    }
    *out = static_cast<int32_t*>(p);
    return FSI_OK;
}

}  // namespace

}  // namespace fsi

using namespace fsi;

extern "C" fsi_status fsi_batched_lu_noalloc(int precision, int batch, int m, int ncols, int npiv, void* A,
                                             int64_t ld, int64_t sA, int32_t* ipiv, int* n_singular_out,
                                             void* stream) {
    if (!(A && ipiv && batch > 0 && m > 0 && ncols > 0)) {
        set_error("fsi_batched_lu_noalloc: bad arguments");
        return FSI_EINVAL;
    }
    if (!(npiv > 0 && npiv <= m && npiv <= ncols && ld >= ncols && sA >= ld * m)) {
        set_error("fsi_batched_lu_noalloc: bad shape");
        return FSI_EINVAL;
    }
    if (precision == FSI_BF16X6_IR || precision == FSI_BF16_IR) {
        set_error("fsi_batched_lu_noalloc: the tensor-core precisions need an operand workspace; use fsi_batched_lu");
        return FSI_EINVAL;
    }
    if (precision != FSI_FP64 && precision != FSI_FP32_IR) {
        set_error("fsi_batched_lu_noalloc: unknown precision");
        return FSI_EINVAL;
    }
    if (batch > kNoAllocMaxBatch) {
        std::ostringstream o;
        o << "fsi_batched_lu_noalloc: batch " << batch << " exceeds the built-in scratch limit of "
          << kNoAllocMaxBatch << " matrices; split the call or use fsi_batched_lu with a workspace";
        set_error(o.str());
        return FSI_EINVAL;
    }
    if (m > 8192) {
        set_error("fsi_batched_lu_noalloc: m too large for the panel kernel");
        return FSI_EINVAL;
    }
    int32_t* scratch = nullptr;
    fsi_status s = scratch_for_current_device(&scratch);
    if (s != FSI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // flags must start at zero; the counter too
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int32_t) * batch, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + kNoAllocMaxBatch, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        return FSI_ECUDA;
    }
    if (precision == FSI_FP64)
        partial_lu<double>(static_cast<double2*>(A), sA, int(ld), batch, m, ncols, npiv, ipiv, npiv, scratch, st);
    else
        partial_lu<float>(static_cast<float2*>(A), sA, int(ld), batch, m, ncols, npiv, ipiv, npiv, scratch, st,
                          nullptr);
    count_flags_kernel<<<1, 256, 0, st>>>(scratch, batch, scratch + kNoAllocMaxBatch);
    e = cudaGetLastError();
    if (e == cudaSuccess && n_singular_out) {
        int32_t cnt = 0;
        e = cudaMemcpyAsync(&cnt, scratch + kNoAllocMaxBatch, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        *n_singular_out = cnt;
    }
    if (e != cudaSuccess) {
        set_error(std::string("fsi_batched_lu_noalloc: ") + cudaGetErrorString(e));
        return FSI_ECUDA;
    }
    return FSI_OK;
}

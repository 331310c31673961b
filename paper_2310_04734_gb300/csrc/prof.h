// Optional per-kernel CUDA-event timing of the launches made by one API call.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace fsi {

enum ProfKind { PK_GEMM = 0, PK_PANEL, PK_TRSM, PK_LASWP, PK_FORM, PK_SHIFT, PK_SOLVE, PK_RESID, PK_GEMV, PK_PACK, PK_TCGEMM, PK_COUNT };

struct ProfRec {
    int kind;
    cudaEvent_t a, b;
    double flops;
};

struct Prof {
    bool on = false;
    int64_t launches = 0;
    std::vector<cudaEvent_t> pool;
    std::vector<ProfRec> recs;
    double ms[PK_COUNT] = {0};
    double flops[PK_COUNT] = {0};
    int64_t count[PK_COUNT] = {0};
    void reset(bool enable);
    cudaEvent_t event();
    // fold recorded event pairs into the totals (the stream must have been synchronized)
    void collect();
};

Prof& prof();

// Counts one launch and, when profiling is on, brackets it with events on `st`.
struct ProfScope {
    int kind;
    double flops;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(int k, double f, cudaStream_t s);
    ~ProfScope();
};

}  // namespace fsi

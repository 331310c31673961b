#include "prof.h"

namespace fsi {

Prof& prof() {
    static thread_local Prof p;
    return p;
}

void Prof::reset(bool enable) {
    for (auto& r : recs) {
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
    on = enable;
    launches = 0;
    for (int i = 0; i < PK_COUNT; ++i) {
        ms[i] = 0.0;
        flops[i] = 0.0;
        count[i] = 0;
    }
}

cudaEvent_t Prof::event() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void Prof::collect() {
    for (auto& r : recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.kind] += t;
        flops[r.kind] += r.flops;
        count[r.kind] += 1;
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

ProfScope::ProfScope(int k, double f, cudaStream_t s) : kind(k), flops(f), st(s) {
    Prof& p = prof();
    p.launches += 1;
    if (p.on) {
        a = p.event();
        cudaEventRecord(a, st);
    }
}

ProfScope::~ProfScope() {
    Prof& p = prof();
    if (p.on && a) {
        cudaEvent_t b = p.event();
        cudaEventRecord(b, st);
        p.recs.push_back(ProfRec{kind, a, b, flops});
    }
}

}  // namespace fsi

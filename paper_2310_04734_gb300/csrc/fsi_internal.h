// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fsi.h"

namespace fsi {

// Thread-local error message behind fsi_last_error().
void set_error(const std::string& msg);

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of the arrays inside the device model buffer.
struct ModelLayout {
    size_t rowptr, col, K, M, D, kdiag, cbase, rbase, total;
};
ModelLayout model_layout(const fsi_dims& d);

// Host-side assembled model (CSR with a shared pattern).
struct HostModel {
    fsi_dims dims{};
    std::vector<int32_t> rowptr, col;
    std::vector<fsi_c64> K, D;
    std::vector<double> M;
    std::vector<double> kdiag;  // |K_ii|
};
fsi_status assemble_host(const fsi_model_desc& desc, HostModel& out);
fsi_status validate_desc(const fsi_model_desc& desc);

// Carves aligned sub-buffers out of a caller-provided workspace.
struct Carver {
    char* base;
    size_t used = 0, cap;
    Carver(void* p, size_t c) : base(static_cast<char*>(p)), cap(c) {}
    template <typename T>
    T* take(size_t count) {
        size_t off = align_up(used);
        used = off + count * sizeof(T);
        return base ? reinterpret_cast<T*>(base + off) : nullptr;
    }
    bool fits() const { return used <= cap; }
};

}  // namespace fsi

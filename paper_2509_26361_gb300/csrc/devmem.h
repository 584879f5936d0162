// Device allocations of the library: cudaMalloc/cudaFree, or the caller's
// allocator installed with ebit_set_allocator.  Each object (context,
// network, batch) takes a copy of the allocator in force when it is created
// and frees everything it allocated through that copy, so replacing the
// allocator later never pairs one allocator's pointer with another's free.
#pragma once
#include <cuda_runtime.h>

#include "ebit.h"

namespace ebit {

struct DevMem {
    ebit_alloc_fn alloc = nullptr;  // null: cudaMalloc / cudaFree
    ebit_free_fn free = nullptr;
    void *user = nullptr;
};

// the allocator in force (defined in ebit_abi.cu)
DevMem current_devmem();

inline bool dev_alloc(const DevMem &m, void **p, size_t bytes) {
    if (m.alloc) {
        *p = m.alloc(bytes, m.user);
        return *p != nullptr;
    }
    return cudaMalloc(p, bytes) == cudaSuccess;
}

inline void dev_free(const DevMem &m, void *p) {
    if (!p) return;
    if (m.free)
        m.free(p, m.user);
    else
        cudaFree(p);
}

}  // namespace ebit

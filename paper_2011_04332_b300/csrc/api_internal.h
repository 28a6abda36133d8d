// Library-internal definitions shared by the translation units of libnpfem.so.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/npfem.h"
#include "npfem_internal.h"

namespace npfem {

// Device allocation list owned by a type or batch.
struct DevAllocs {
  std::vector<void*> ptrs;
  ~DevAllocs() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  cudaError_t upload(const std::vector<T>& h, const T** out) {
    void* d = nullptr;
    size_t bytes = std::max<size_t>(1, h.size()) * sizeof(T);
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return e;
    ptrs.push_back(d);
    if (!h.empty()) e = cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    *out = static_cast<const T*>(d);
    return e;
  }
  cudaError_t alloc(size_t bytes, void** out) {
    cudaError_t e = cudaMalloc(out, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) ptrs.push_back(*out);
    return e;
  }
};

}  // namespace npfem

struct npfem_cell_type {
  npfem::HostType host;
  npfem::DevAllocs mem;
  npfem::DevTypeView<double> v64;
  npfem::DevTypeView<float> v32;
  int device = 0;
};

// Record `msg` as the calling thread's last error and return `code`.
npfem_status npfem_internal_fail(npfem_status code, const std::string& msg);

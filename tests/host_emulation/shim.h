// Host compilation shim: lets g++ compile the library's device code (FP64
// kernels without inline PTX) so a CPU test can run each kernel body once per
// emulated thread and compare the result with the oracle.  Only what those
// kernels use is provided; anything else fails to compile or link.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>

struct EmuDim {
  unsigned x, y, z;
};
extern EmuDim blockIdx, threadIdx, blockDim, gridDim;

template <typename T>
inline T __ldg(const T* p) { return *p; }
inline int atomicOr(int* p, int v) { const int o = *p; *p |= v; return o; }
inline unsigned __umulhi(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }
inline size_t __cvta_generic_to_shared(const void* p) { return (size_t)p; }
inline void __syncthreads() {}  // the emulated kernels are run without their CTA reductions
#define __launch_bounds__(...)
using std::fma;
using std::isnan;

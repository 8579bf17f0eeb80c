// Launch forms of the library's host code on the threaded emulator: the
// triple-chevron launches and cudaLaunchKernelEx (with its cluster
// dimension) become emu_launch3 calls that run the kernel to completion.
#pragma once

inline dim3 emu_dim(dim3 d) { return d; }
inline dim3 emu_dim(unsigned v) { return dim3(v, 1, 1); }
inline dim3 emu_dim(int v) { return dim3((unsigned)v, 1, 1); }
inline dim3 emu_dim(long long v) { return dim3((unsigned)v, 1, 1); }

template <typename G, typename B, typename F>
void emu_kernel_launch(G grid, B block, size_t smem, cudaStream_t, F body) {
  const dim3 gd = emu_dim(grid), bd = emu_dim(block);
  if (gd.x == 0) return;
  emu_launch3((int)(gd.x * gd.y * gd.z), 1, bd, smem, body);
}

template <typename... P, typename... A>
cudaError_t emu_launch_ex(const cudaLaunchConfig_t* cfg, void (*kernel)(P...), A&&... args) {
  int cs = 1;
  for (unsigned i = 0; i < cfg->numAttrs; ++i)
    if (cfg->attrs[i].id == cudaLaunchAttributeClusterDimension) cs = (int)cfg->attrs[i].val.clusterDim.x;
  const int nclusters = (int)(cfg->gridDim.x / cs);
  emu_launch3(nclusters, cs, cfg->blockDim, cfg->dynamicSmemBytes, [&] { kernel(args...); });
  return cudaSuccess;
}

// the typed forms the CUDA headers provide to nvcc only
template <typename... P>
cudaError_t cudaFuncSetAttribute(void (*k)(P...), enum cudaFuncAttribute a, int v) {
  return cudaFuncSetAttribute(reinterpret_cast<const void*>(k), a, v);
}
template <typename... P>
cudaError_t cudaOccupancyMaxActiveClusters(int* n, void (*k)(P...), const cudaLaunchConfig_t* c) {
  return cudaOccupancyMaxActiveClusters(n, reinterpret_cast<const void*>(k), c);
}

// the device-side setter of a conditional graph node's value (the emulated
// runtime refuses to build such graphs, so it is never reached)
inline void cudaGraphSetConditional(cudaGraphConditionalHandle, unsigned int) {}

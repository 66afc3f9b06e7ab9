// TEST INFRASTRUCTURE: host-only stand-ins for the CUDA runtime calls the
// library's host code makes.  "Device" memory is host memory and copies are
// memcpy.  Used by the host-ABI harness and by the CPU emulation of the
// kernels; the product library never links it.
#include <cuda_runtime_api.h>

#include <cstring>

extern "C" {

cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaGetDevice(int* d) {
  *d = 0;
  return cudaSuccess;
}
cudaError_t cudaFuncSetAttribute(const void*, enum cudaFuncAttribute, int) { return cudaSuccess; }
// One SM: in the CPU emulation a batch of two or more binary32 chains takes
// the two-chains-per-SM kernel, a single chain the one-chain kernel.
cudaError_t cudaDeviceGetAttribute(int* value, enum cudaDeviceAttr attr, int) {
  *value = attr == cudaDevAttrMultiProcessorCount ? 1 : 0;
  return cudaSuccess;
}
cudaError_t cudaGetSymbolAddress(void** p, const void* symbol) {
  *p = const_cast<void*>(symbol);
  return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
const char* cudaGetErrorString(cudaError_t) { return "stub"; }
cudaError_t cudaMemcpy(void* dst, const void* src, size_t n, enum cudaMemcpyKind) {
  std::memmove(dst, src, n);
  return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void* dst, const void* src, size_t n, enum cudaMemcpyKind, cudaStream_t) {
  std::memmove(dst, src, n);
  return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void* dst, int v, size_t n, cudaStream_t) {
  std::memset(dst, v, n);
  return cudaSuccess;
}

}  // extern "C"

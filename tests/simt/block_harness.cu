// TEST INFRASTRUCTURE: runs pieces of the library's split (hm_block.cuh) in
// the CPU emulation, so that the tests can check them directly: the
// one-sided Jacobi of one block (jacobi_group) on crafted matrices (graded
// spectra, noise-level columns, exact degeneracy) against numpy, and the
// truncation rule (trunc_rank) against the oracle's.  Built only by
// build_emulated.py; the product library never links it.
#include <vector>

#include "hm_block.cuh"

namespace {

__global__ void jacobi_probe64(double* W, int q, int p, double* V, double* nrm, double stop, int* sweeps) {
  __shared__ hm::blk::GroupSh gs;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // the binary64 kernels' batch of two rows per lane
  const int s = hm::blk::jacobi_group<double, double, 2>(W, q, q, p, V, p, nrm, warp, nw, 1, 0, gs, stop, 60);
  if (threadIdx.x == 0) *sweeps = s;
}

__global__ void jacobi_probe32(float* W, int q, int p, float* V, float* nrm, float stop, int* sweeps) {
  __shared__ hm::blk::GroupSh gs;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int s = hm::blk::jacobi_group<float>(W, q, q, p, V, p, nrm, warp, nw, 1, 0, gs, stop, 60);
  if (threadIdx.x == 0) *sweeps = s;
}

}  // namespace

// W: q x p column-major (q >= p), V: p x p column-major holding the starting
// basis; both overwritten.  Binary64 when binary64 != 0, else binary32.
// Returns the sweeps, or -1 when 60 sweeps did not converge.
extern "C" int hm_probe_jacobi(void* W, int q, int p, void* V, int binary64, int nthreads, double stop) {
  int sweeps = 0;
  if (binary64) {
    std::vector<double> nrm(p);
    jacobi_probe64<<<1, nthreads, 0, nullptr>>>((double*)W, q, p, (double*)V, nrm.data(), stop, &sweeps);
  } else {
    std::vector<float> nrm(p);
    jacobi_probe32<<<1, nthreads, 0, nullptr>>>((float*)W, q, p, (float*)V, nrm.data(), (float)stop, &sweeps);
  }
  return sweeps;
}

// Kept count of the truncation rule for n descending values s (the
// device function itself, called on the host in the emulation).  tail and
// total are outputs (tail: n + 1 doubles).
extern "C" int hm_probe_trunc(const double* s, int n, int chi_max, double cutoff, double* tail, double* total) {
  return hm::blk::trunc_rank(s, n, chi_max, cutoff, tail, total);
}

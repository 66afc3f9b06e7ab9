// The mixed-precision evolve kernel of hm_mixed.cu built for two CTAs per
// SM: 256 threads and 108 KB of shared memory each.  launch_evolve_mixed
// sends a batch here when it has more chains than the GPU has SMs and its
// bond cap keeps the charge blocks within 108 KB: every chain of the batch is
// then resident at once (152 SMs hold 304 chains instead of 152), and each
// SM interleaves two independent chains, whose Jacobi rounds wait at their
// own barriers.
#define HM_MIXED_NT 256
#define HM_MIXED_CTAS_PER_SM 2
#include "hm_mixed.cu"

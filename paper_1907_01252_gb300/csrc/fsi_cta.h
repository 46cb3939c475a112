// A cooperative thread group for routines written once for the device and the
// host: a CUDA block (DevCta: threadIdx.x of blockDim.x, sync = __syncthreads)
// or one host thread (HostCta: the same phases in the same order, sync = no-op).
#pragma once

#ifdef __CUDACC__
#define FSI_CTA_HD __host__ __device__
#else
#define FSI_CTA_HD
#endif

namespace fsi3 {

struct HostCta {
  int tid = 0, nt = 1;
  FSI_CTA_HD void sync() const {}
};
#ifdef __CUDACC__
struct DevCta {
  int tid, nt;
  __device__ void sync() const { __syncthreads(); }
};
#endif

}  // namespace fsi3

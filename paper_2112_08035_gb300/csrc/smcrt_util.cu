// smcrt_util.cu -- small helper kernels of the runtime.
#include "smcrt_internal.h"

namespace smcrt {

namespace {

// Writes a job descriptor into device memory.  Passing it as a kernel
// parameter captures its value at launch time, so consecutive launches on
// a stream (or inside a CUDA graph) never race on a host staging buffer.
__global__ void set_jobs_kernel(JobWork *dst, JobWork v) { *dst = v; }

}  // namespace

cudaError_t launch_set_job(JobWork *dst, const JobWork &v, cudaStream_t stream)
{
    set_jobs_kernel<<<1, 1, 0, stream>>>(dst, v);
    return cudaGetLastError();
}

}  // namespace smcrt

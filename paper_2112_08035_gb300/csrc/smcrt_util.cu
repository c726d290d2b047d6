// smcrt_util.cu -- small helper kernels of the runtime.
#include "smcrt_internal.h"

namespace smcrt {

namespace {

// Writes a job descriptor into device memory.  Passing it as a kernel
// parameter captures its value at launch time, so consecutive launches on
// a stream (or inside a CUDA graph) never race on a host staging buffer.
__global__ void set_jobs_kernel(JobWork *dst, JobWork v) { *dst = v; }

__global__ void round_prologue_kernel(JobWork *jobs, int njobs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= njobs) return;
    JobDefer *d = jobs[i].defer;
    if (d == nullptr) return;
    const int in = jobs[i].defer_in & 1;
    d->cursor[in] = 0u;
    d->count[1 - in] = 0u;
    d->cursor[1 - in] = 0u;
}

}  // namespace

cudaError_t launch_round_prologue(JobWork *jobs, int njobs, cudaStream_t stream)
{
    round_prologue_kernel<<<(njobs + 127) / 128, 128, 0, stream>>>(jobs, njobs);
    return cudaGetLastError();
}

cudaError_t launch_set_job(JobWork *dst, const JobWork &v, cudaStream_t stream)
{
    set_jobs_kernel<<<1, 1, 0, stream>>>(dst, v);
    return cudaGetLastError();
}

}  // namespace smcrt

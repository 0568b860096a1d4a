// k_common.cu -- kernels shared by every parameter set: message offsets.
#include <cuda_runtime.h>
#include "hs_launch.h"

namespace hs {

// ------------------------------------------------------------- offsets
// offsets[i] = lens[0] + ... + lens[i-1], i = 0..count (one CTA of 1024).
__global__ void offsets_kernel(const uint64_t* __restrict__ lens, uint32_t count, uint64_t* __restrict__ off) {
    __shared__ uint64_t part[1024];
    const uint32_t t = threadIdx.x;
    const uint32_t chunk = (count + 1023) / 1024;
    const uint64_t lo = (uint64_t)t * chunk;
    uint64_t s = 0;
    for (uint64_t i = lo; i < lo + chunk && i < count; i++) s += lens[i];
    part[t] = s;
    __syncthreads();
    for (uint32_t d = 1; d < 1024; d <<= 1) {       // inclusive Hillis-Steele scan
        uint64_t v = (t >= d) ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint64_t run = (t == 0) ? 0 : part[t - 1];
    for (uint64_t i = lo; i < lo + chunk && i < count; i++) { off[i] = run; run += lens[i]; }
    if (t == 1023) off[count] = part[1023];
}

cudaError_t launch_offsets(const Batch& b, cudaStream_t s) {
    offsets_kernel<<<1, 1024, 0, s>>>(b.lens, b.count, b.offsets);
    return cudaGetLastError();
}

}  // namespace hs

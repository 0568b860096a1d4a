// probe.cu -- measured integer-pipe rates of the current GPU, for the
// roofline that bench.py reports (the signer itself never calls this).
//
// Each probe kernel runs independent streams of one instruction form (8
// accumulators per thread, so no dependency stalls) on full-occupancy
// blocks.  Every block records its SM id and its elapsed SM cycles; the
// rate of an SM is the lane-operations of its blocks divided by the longest
// of their cycle counts, averaged over SMs.  Results are in lane-ops per
// clock per SM, so they do not depend on the clock the GPU happened to run at.
#include <cuda_runtime.h>
#include <cstdint>
#include <vector>
#include "../../include/hs.h"

#define HS_API extern "C" __attribute__((visibility("default")))

namespace hs {
namespace {

#define P_LOP3(x, y, z) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x) : "r"(y), "r"(z))
#define P_SHF(x) asm volatile("shf.r.wrap.b32 %0, %0, %0, 7;" : "+r"(x))
#define P_ADD(x, y) asm volatile("add.u32 %0, %0, %1;" : "+r"(x) : "r"(y))
#define P_MAD(x, one, y) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(one), "r"(y))
#define P_MADHI(x, m, y) asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x) : "r"(m), "r"(y))
#define P_PRMT(x, y) asm volatile("prmt.b32 %0, %0, %1, 0x5432;" : "+r"(x) : "r"(y))

// OP: 0 LOP3, 1 SHF, 2 IADD, 3 IMAD, 4 IMAD.HI, 5 PRMT, 6 LOP3+IMAD
template <int OP>
__global__ void __launch_bounds__(256) pipe_probe(int iters, uint32_t one, uint32_t seed, uint32_t* sink,
                                                  long long* cyc, int* smid) {
    uint32_t a[8];
    const uint32_t y = seed ^ threadIdx.x, z = seed * 3u;
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = seed + i * 977u + threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (OP == 0) { P_LOP3(a[i], y, z); P_LOP3(a[i], z, y); }
            if (OP == 1) { P_SHF(a[i]); P_SHF(a[i]); }
            if (OP == 2) { P_ADD(a[i], y); P_ADD(a[i], z); }
            if (OP == 3) { P_MAD(a[i], one, y); P_MAD(a[i], one, z); }
            if (OP == 4) { P_MADHI(a[i], one, y); P_MADHI(a[i], one, z); }
            if (OP == 5) { P_PRMT(a[i], y); P_PRMT(a[i], z); }
            if (OP == 6) { P_LOP3(a[i], y, z); P_MAD(a[i], one, z); }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) s ^= a[i];
    if (s == 0x12345678u) sink[0] = s;       // keeps the work alive; practically never stores
    if (threadIdx.x == 0) {
        cyc[blockIdx.x] = t1 - t0;
        int id;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
        smid[blockIdx.x] = id;
    }
}

template <int OP>
cudaError_t run_probe(int blocks, int iters, uint32_t* sink, long long* cyc, int* smid) {
    pipe_probe<OP><<<blocks, 256>>>(iters, 1u, 7u, sink, cyc, smid);
    return cudaGetLastError();
}

}  // namespace
}  // namespace hs

using namespace hs;

// Rates of the 7 forms (see the OP list above) in lane-ops / clock / SM.
// Synchronizes the device; allocates and frees a small device buffer.
// Returns the number of rates written (<= max) or -1 on a CUDA error.
HS_API int hs_probe_int_pipes(float* rates, int max) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    const int blocks = sms * 8, iters = 2048;
    uint32_t* sink = nullptr;
    long long* cyc = nullptr;
    int* smid = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return -1;
    if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) { cudaFree(sink); return -1; }
    if (cudaMalloc(&smid, sizeof(int) * blocks) != cudaSuccess) { cudaFree(sink); cudaFree(cyc); return -1; }
    std::vector<long long> hc(blocks);
    std::vector<int> hs(blocks);
    int n = 0;
    cudaError_t e = cudaSuccess;
    for (int op = 0; op < 7 && n < max; op++) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {   // first run warms up
            switch (op) {
            case 0: e = run_probe<0>(blocks, iters, sink, cyc, smid); break;
            case 1: e = run_probe<1>(blocks, iters, sink, cyc, smid); break;
            case 2: e = run_probe<2>(blocks, iters, sink, cyc, smid); break;
            case 3: e = run_probe<3>(blocks, iters, sink, cyc, smid); break;
            case 4: e = run_probe<4>(blocks, iters, sink, cyc, smid); break;
            case 5: e = run_probe<5>(blocks, iters, sink, cyc, smid); break;
            case 6: e = run_probe<6>(blocks, iters, sink, cyc, smid); break;
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e != cudaSuccess) break;
        cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
        cudaMemcpy(hs.data(), smid, sizeof(int) * blocks, cudaMemcpyDeviceToHost);
        std::vector<long long> maxc(1024, 0);
        std::vector<int> nblk(1024, 0);
        for (int b = 0; b < blocks; b++) {
            const int s = hs[b] & 1023;
            if (hc[b] > maxc[s]) maxc[s] = hc[b];
            nblk[s]++;
        }
        const double ops_per_block = 256.0 * iters * 8 * 2;
        double sum = 0;
        int used = 0;
        for (int s = 0; s < 1024; s++)
            if (nblk[s] && maxc[s] > 0) { sum += ops_per_block * nblk[s] / (double)maxc[s]; used++; }
        rates[n++] = used ? (float)(sum / used) : 0.f;
    }
    cudaFree(sink);
    cudaFree(cyc);
    cudaFree(smid);
    return e == cudaSuccess ? n : -1;
}

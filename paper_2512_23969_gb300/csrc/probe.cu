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
#include "sha2.cuh"
#include "sha256_chain.cuh"

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

// SHA-2 mix probes: the signer's own compression functions, run back to
// back on an independent state per thread (a thread's next block is built
// from its last result, so nothing is loop-invariant).  The rate is
// compressions per clock per SM: the ceiling the SHA-2 instruction mix
// itself reaches on this GPU, carry pairs and all, with no kernel overhead.
// KIND 0: SHA-256 with the signer's round code (all 64 rounds unrolled,
//         round additions on IMAD: Rounds256 with the chain policy);
// KIND 1: SHA-512, 16 rounds in a loop of 5 (sha512_compress);
// KIND 2: 64-bit additions (add.u64, two 32-bit halves with a carry);
// KIND 3: SHA-256 as FIPS 180-4 writes it (sha256_compress_full).
template <int KIND>
__global__ void __launch_bounds__(256) sha_probe(int iters, uint32_t seed, uint32_t one, uint32_t* sink,
                                                 long long* cyc, int* smid) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t s = 0;
    __syncthreads();
    const long long t0 = clock64();
    if constexpr (KIND == 0) {
        const Pipes<kChainPol> pp(one);
        uint32_t st[8];
#pragma unroll
        for (int i = 0; i < 8; i++) st[i] = seed * (2u * i + 1u) + tid;
        for (int it = 0; it < iters; it++) {
            uint32_t W[16], v[8];
#pragma unroll
            for (int i = 0; i < 8; i++) { W[i] = st[i]; W[i + 8] = st[i] + 0x9e3779b9u * (i + 1); v[i] = st[i]; }
            Rounds256<kChainPol, false, 0, 64>::run(v, W, nullptr, pp);
#pragma unroll
            for (int i = 0; i < 8; i++) st[i] += v[i];
        }
#pragma unroll
        for (int i = 0; i < 8; i++) s ^= st[i];
    } else if constexpr (KIND == 3) {
        uint32_t st[8];
#pragma unroll
        for (int i = 0; i < 8; i++) st[i] = seed * (2u * i + 1u) + tid;
        for (int it = 0; it < iters; it++) {
            uint32_t W[16];
#pragma unroll
            for (int i = 0; i < 8; i++) { W[i] = st[i]; W[i + 8] = st[i] + 0x9e3779b9u * (i + 1); }
            sha256_compress_full(st, W);
        }
#pragma unroll
        for (int i = 0; i < 8; i++) s ^= st[i];
    } else if constexpr (KIND == 1) {
        uint64_t st[8];
#pragma unroll
        for (int i = 0; i < 8; i++) st[i] = ((uint64_t)(seed * (2u * i + 1u)) << 32) | (tid + i);
        for (int it = 0; it < iters; it++) {
            uint64_t W[16];
#pragma unroll
            for (int i = 0; i < 8; i++) { W[i] = st[i]; W[i + 8] = st[i] + 0x9e3779b97f4a7c15ull * (i + 1); }
            sha512_compress(st, W);
        }
#pragma unroll
        for (int i = 0; i < 8; i++) s ^= (uint32_t)st[i] ^ (uint32_t)(st[i] >> 32);
    } else {
        uint64_t a[8];
        const uint64_t y = ((uint64_t)seed << 32) | (tid * 3u + 1u), z = y * 5u + 0x100000001ull;
#pragma unroll
        for (int i = 0; i < 8; i++) a[i] = y * (i + 7u);
        for (int it = 0; it < iters; it++) {
#pragma unroll
            for (int i = 0; i < 8; i++) {
                asm volatile("add.u64 %0, %0, %1;" : "+l"(a[i]) : "l"(y));
                asm volatile("add.u64 %0, %0, %1;" : "+l"(a[i]) : "l"(z));
            }
        }
#pragma unroll
        for (int i = 0; i < 8; i++) s ^= (uint32_t)a[i] ^ (uint32_t)(a[i] >> 32);
    }
    __syncthreads();
    const long long t1 = clock64();
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

template <int KIND>
cudaError_t run_sha_probe(int blocks, int iters, uint32_t* sink, long long* cyc, int* smid) {
    sha_probe<KIND><<<blocks, 256>>>(iters, 0x2512u, 1u, sink, cyc, smid);
    return cudaGetLastError();
}

// Per-SM rate from one launch: the operations of an SM's blocks divided by
// the longest of their cycle counts (all blocks of a launch are resident
// at once), averaged over the SMs that ran blocks.
float sm_rate(const std::vector<long long>& hc, const std::vector<int>& hs, double ops_per_block) {
    std::vector<long long> maxc(1024, 0);
    std::vector<int> nblk(1024, 0);
    for (size_t b = 0; b < hc.size(); b++) {
        const int s = hs[b] & 1023;
        if (hc[b] > maxc[s]) maxc[s] = hc[b];
        nblk[s]++;
    }
    double sum = 0;
    int used = 0;
    for (int s = 0; s < 1024; s++)
        if (nblk[s] && maxc[s] > 0) { sum += ops_per_block * nblk[s] / (double)maxc[s]; used++; }
    return used ? (float)(sum / used) : 0.f;
}

struct ProbeBufs {
    uint32_t* sink = nullptr;
    long long* cyc = nullptr;
    int* smid = nullptr;
    bool alloc(int blocks) {
        return cudaMalloc(&sink, 64) == cudaSuccess && cudaMalloc(&cyc, sizeof(long long) * blocks) == cudaSuccess &&
               cudaMalloc(&smid, sizeof(int) * blocks) == cudaSuccess;
    }
    ~ProbeBufs() {
        if (sink) cudaFree(sink);
        if (cyc) cudaFree(cyc);
        if (smid) cudaFree(smid);
    }
    bool read(int blocks, std::vector<long long>& hc, std::vector<int>& hs) const {
        hc.resize(blocks);
        hs.resize(blocks);
        return cudaMemcpy(hc.data(), cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost) == cudaSuccess &&
               cudaMemcpy(hs.data(), smid, sizeof(int) * blocks, cudaMemcpyDeviceToHost) == cudaSuccess;
    }
};

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
    ProbeBufs pb;
    if (!pb.alloc(blocks)) { cudaGetLastError(); return -1; }
    std::vector<long long> hc;
    std::vector<int> hs;
    int n = 0;
    cudaError_t e = cudaSuccess;
    for (int op = 0; op < 7 && n < max; op++) {
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {   // first run warms up
            switch (op) {
            case 0: e = run_probe<0>(blocks, iters, pb.sink, pb.cyc, pb.smid); break;
            case 1: e = run_probe<1>(blocks, iters, pb.sink, pb.cyc, pb.smid); break;
            case 2: e = run_probe<2>(blocks, iters, pb.sink, pb.cyc, pb.smid); break;
            case 3: e = run_probe<3>(blocks, iters, pb.sink, pb.cyc, pb.smid); break;
            case 4: e = run_probe<4>(blocks, iters, pb.sink, pb.cyc, pb.smid); break;
            case 5: e = run_probe<5>(blocks, iters, pb.sink, pb.cyc, pb.smid); break;
            case 6: e = run_probe<6>(blocks, iters, pb.sink, pb.cyc, pb.smid); break;
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e != cudaSuccess || !pb.read(blocks, hc, hs)) break;
        rates[n++] = sm_rate(hc, hs, 256.0 * iters * 8 * 2);
    }
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess ? n : -1;
}

// SHA-2 mix rates: 0 SHA-256 compressions (the signer's round code), 1
// SHA-512 compressions, per clock per SM; 2 64-bit additions in lane-ops
// per clock per SM; 3 SHA-256 compressions as FIPS 180-4 writes them.  Each
// probe's grid is one wave of its occupancy limit.  Synchronizes the
// device; allocates and frees a small device buffer.  Returns the number
// of rates written (<= max) or -1 on a CUDA error.
HS_API int hs_probe_sha_mix(float* rates, int max) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    constexpr int kKinds = 4;
    int per_sm[kKinds] = {0, 0, 0, 0};
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], sha_probe<0>, 256, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], sha_probe<1>, 256, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2], sha_probe<2>, 256, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[3], sha_probe<3>, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    const int iters[kKinds] = {96, 32, 2048, 96};
    const double ops[kKinds] = {256.0 * iters[0], 256.0 * iters[1], 256.0 * iters[2] * 8 * 2, 256.0 * iters[3]};
    int maxb = 0;
    for (int k = 0; k < kKinds; k++) {
        if (per_sm[k] < 1) per_sm[k] = 1;
        if (sms * per_sm[k] > maxb) maxb = sms * per_sm[k];
    }
    ProbeBufs pb;
    if (!pb.alloc(maxb)) { cudaGetLastError(); return -1; }
    std::vector<long long> hc;
    std::vector<int> hs;
    int n = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kKinds && n < max; k++) {
        const int blocks = sms * per_sm[k];
        for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {   // first run warms up
            switch (k) {
            case 0: e = run_sha_probe<0>(blocks, iters[k], pb.sink, pb.cyc, pb.smid); break;
            case 1: e = run_sha_probe<1>(blocks, iters[k], pb.sink, pb.cyc, pb.smid); break;
            case 2: e = run_sha_probe<2>(blocks, iters[k], pb.sink, pb.cyc, pb.smid); break;
            case 3: e = run_sha_probe<3>(blocks, iters[k], pb.sink, pb.cyc, pb.smid); break;
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e != cudaSuccess || !pb.read(blocks, hc, hs)) break;
        rates[n++] = sm_rate(hc, hs, ops[k]);
    }
    if (e != cudaSuccess) cudaGetLastError();
    return e == cudaSuccess ? n : -1;
}

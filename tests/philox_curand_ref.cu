// Test helper: Philox4x32-10 outputs from cuRAND's device generator
// (curandStatePhilox4_32_10_t), an implementation independent of both the
// oracle and the library.  curand_init(seed, subsequence, offset) places the
// 128-bit counter at (offset / 4) + 2^64 * subsequence under key = seed, and
// curand4 returns the block at that counter.  Built and loaded by the tests.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_curand_blocks(const unsigned long long* seed, const unsigned long long* subseq,
                                const unsigned long long* offset, uint32_t* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed[i], subseq[i], offset[i], &st);
    const uint4 v = curand4(&st);
    out[4 * i + 0] = v.x;
    out[4 * i + 1] = v.y;
    out[4 * i + 2] = v.z;
    out[4 * i + 3] = v.w;
}

extern "C" int curand_philox_blocks(const unsigned long long* seed, const unsigned long long* subseq,
                                    const unsigned long long* offset, uint32_t* out, int n) {
    unsigned long long *ds = nullptr, *dq = nullptr, *doff = nullptr;
    uint32_t* dout = nullptr;
    const size_t b8 = sizeof(unsigned long long) * (size_t)n;
    if (cudaMalloc(&ds, b8) || cudaMalloc(&dq, b8) || cudaMalloc(&doff, b8) ||
        cudaMalloc(&dout, 16 * (size_t)n))
        return 1;
    cudaMemcpy(ds, seed, b8, cudaMemcpyHostToDevice);
    cudaMemcpy(dq, subseq, b8, cudaMemcpyHostToDevice);
    cudaMemcpy(doff, offset, b8, cudaMemcpyHostToDevice);
    k_curand_blocks<<<(n + 127) / 128, 128>>>(ds, dq, doff, dout, n);
    const int err = (int)cudaMemcpy(out, dout, 16 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(ds);
    cudaFree(dq);
    cudaFree(doff);
    cudaFree(dout);
    return err;
}

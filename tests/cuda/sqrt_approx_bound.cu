// Measures the relative error of the PTX sqrt.approx.ftz.f32 instruction
// against the correctly rounded FP32 square root (sqrt.rn.f32) at every float
// in [2^-37, 2^15) and prints the maximum relative error.  That range holds
// every positive variance the window kernels can form: V / n^2 >= 1 / n^2 >=
// 1 / 511^4 > 2^-37 and V / n^2 <= 255^2 / 4 < 2^14 (with rounding to spare).
// The kernels' certified FP32 threshold bound assumes at most 2^-22.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__global__ void k(uint32_t lo, uint32_t hi, uint32_t step, unsigned long long *worst_bits)
{
    double worst = 0.0;
    for (uint64_t b = (uint64_t)lo + (uint64_t)(blockIdx.x * blockDim.x + threadIdx.x) * step; b < hi;
         b += (uint64_t)gridDim.x * blockDim.x * step) {
        const float x = __uint_as_float((uint32_t)b);
        float a, e;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(a) : "f"(x));
        asm("sqrt.rn.f32 %0, %1;" : "=f"(e) : "f"(x));
        const double rel = fabs((double)a - (double)e) / (double)e;
        worst = rel > worst ? rel : worst;
    }
    atomicMax(worst_bits, (unsigned long long)__double_as_longlong(worst));
}

int main()
{
    unsigned long long *d = nullptr, h = 0;
    if (cudaMalloc(&d, 8) != cudaSuccess || cudaMemset(d, 0, 8) != cudaSuccess)
        return 2;
    const uint32_t lo = 0x2D000000u;  // 2^-37
    const uint32_t hi = 0x47000000u;  // 2^15
    k<<<152 * 8, 256>>>(lo, hi, 1u, d);
    if (cudaDeviceSynchronize() != cudaSuccess)
        return 3;
    cudaMemcpy(&h, d, 8, cudaMemcpyDeviceToHost);
    double w;
    memcpy(&w, &h, 8);
    printf("%.9e\n", w);
    cudaFree(d);
    return 0;
}

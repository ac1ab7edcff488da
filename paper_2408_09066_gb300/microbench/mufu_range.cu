// Accuracy of the MUFU sine and cosine (__sincosf) against double precision for
// arguments uniform in [-A, A], A from pi to 128 pi: the absolute error grows
// with the argument (the unit's own range reduction), which decides below what
// phase the encode may feed MUFU unreduced arguments (its tier 0, under 4 turns).
//
// Build and run:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o mufu_range mufu_range.cu && ./mufu_range
#include <cstdio>
#include <cmath>
#include <cuda_runtime.h>
__global__ void k(int n, float amax, float *err_s, float *err_c, unsigned long long seed) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = seed + (unsigned long long)i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull; z = (z ^ (z >> 27)) * 0x94D049BB133111EBull; z ^= z >> 31;
    float u = (float)((z >> 40) * (1.0 / 16777216.0));
    float a = (2.f * u - 1.f) * amax;
    float s, c;
    __sincosf(a, &s, &c);
    double sd = sin((double)a), cd = cos((double)a);
    err_s[i] = (float)fabs((double)s - sd);
    err_c[i] = (float)fabs((double)c - cd);
}
int main() {
    const int n = 1 << 22;
    float *es, *ec; cudaMalloc(&es, n * 4); cudaMalloc(&ec, n * 4);
    float *hs = (float*)malloc(n * 4), *hc = (float*)malloc(n * 4);
    const float pi = 3.14159265358979f;
    float ranges[] = {pi, 2 * pi, 8 * pi, 16 * pi, 32 * pi, 64 * pi, 128 * pi};
    for (float r : ranges) {
        k<<<(n + 255) / 256, 256>>>(n, r, es, ec, 12345ull);
        cudaMemcpy(hs, es, n * 4, cudaMemcpyDeviceToHost);
        cudaMemcpy(hc, ec, n * 4, cudaMemcpyDeviceToHost);
        double ms = 0, mc = 0, as = 0;
        for (int i = 0; i < n; ++i) { ms = fmax(ms, hs[i]); mc = fmax(mc, hc[i]); as += hs[i]; }
        printf("|a| <= %8.3f  max err sin %.3e cos %.3e  mean sin %.3e\n", r, ms, mc, as / n);
    }
    cudaError_t e = cudaGetLastError();
    printf("status %s\n", cudaGetErrorString(e));
    return 0;
}

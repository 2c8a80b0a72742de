// Microbenchmark of GB300 arithmetic rates: FP64 and FP32 FMA throughput and the
// FP64 / FP32 exp(log) evaluation rate.  Standalone (not part of libvfd.so):
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp_rates fp_rates.cu && ./fp_rates
#include <cstdio>
#include <cuda_runtime.h>

template <class T>
__global__ void fma_loop(T *out, int iters, T a, T b)
{
    T x0 = threadIdx.x * 1e-3, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void gamma_loop(double *out, int iters)
{
    double r2 = 0.5 + threadIdx.x * 1e-4, acc = 0.0;
    for (int i = 0; i < iters; ++i) {
        acc += exp(0.1 * r2 - 1.3 * log(r2));
        r2 += 1e-7;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void gamma_loopf(float *out, int iters)
{
    float r2 = 0.5f + threadIdx.x * 1e-4f, acc = 0.0f;
    for (int i = 0; i < iters; ++i) {
        acc += __expf(0.1f * r2 - 1.3f * __logf(r2));
        r2 += 1e-7f;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

int main()
{
    int nb = 152 * 8, nt = 256;
    double *d;
    float *f;
    cudaMalloc(&d, sizeof(double) * nb * nt);
    cudaMalloc(&f, sizeof(float) * nb * nt);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms;
    int it = 4096;
    fma_loop<double><<<nb, nt>>>(d, it, 0.999, 1e-3);
    cudaEventRecord(e0);
    fma_loop<double><<<nb, nt>>>(d, it, 0.999, 1e-3);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp64 fma GFLOP/s %.1f\n", 2.0 * 8 * it * (double)nb * nt / (ms * 1e6));
    it = 65536;
    fma_loop<float><<<nb, nt>>>(f, it, 0.999f, 1e-3f);
    cudaEventRecord(e0);
    fma_loop<float><<<nb, nt>>>(f, it, 0.999f, 1e-3f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp32 fma GFLOP/s %.1f\n", 2.0 * 8 * it * (double)nb * nt / (ms * 1e6));
    it = 256;
    gamma_loop<<<nb, nt>>>(d, it);
    cudaEventRecord(e0);
    gamma_loop<<<nb, nt>>>(d, it);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp64 exp(log) evals/s %.3e\n", it * (double)nb * nt / (ms * 1e-3));
    it = 8192;
    gamma_loopf<<<nb, nt>>>(f, it);
    cudaEventRecord(e0);
    gamma_loopf<<<nb, nt>>>(f, it);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    printf("fp32 __expf(__logf) evals/s %.3e\n", it * (double)nb * nt / (ms * 1e-3));
    printf("err %s\n", cudaGetErrorString(cudaGetLastError()));
    return 0;
}

// Parameter steps (Sec. V-A: gradient descent, or Adam with lr 1e-3), metric
// finalisation and the DFT twiddle table.
#include "common.cuh"
#include "kernels.h"

namespace fdk {

// The gradient enters scaled by gscale (1 for the library's own steps; 1 / ranks for a
// gradient summed over data-parallel ranks).
__global__ void sgd_kernel(long n, float *__restrict__ theta, const float *__restrict__ grad, float lr, float gscale) {
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x)
        theta[j] = fmaf(-lr, gscale * grad[j], theta[j]);
}

// Kingma & Ba: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// theta -= lr (m / c1) / (sqrt(v / c2) + eps), c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void adam_kernel(long n, float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m,
                            float *__restrict__ v, float lr, float c1, float c2, float gscale) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long j = blockIdx.x * (long)blockDim.x + threadIdx.x; j < n; j += (long)gridDim.x * blockDim.x) {
        const float gj = gscale * grad[j];
        const float mj = fmaf(b1, m[j], (1.f - b1) * gj);
        const float vj = fmaf(b2, v[j], (1.f - b2) * gj * gj);
        m[j] = mj;
        v[j] = vj;
        theta[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
    }
}

static unsigned grid_for(long n) {
    long b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t sgd_step(long n, float *theta, const float *grad, float lr, cudaStream_t st, float gscale) {
    sgd_kernel<<<grid_for(n), 256, 0, st>>>(n, theta, grad, lr, gscale);
    return cudaGetLastError();
}

cudaError_t adam_step(long n, float *theta, const float *grad, float *m, float *v, float lr, float c1, float c2,
                      cudaStream_t st, float gscale) {
    adam_kernel<<<grid_for(n), 256, 0, st>>>(n, theta, grad, m, v, lr, c1, c2, gscale);
    return cudaGetLastError();
}

__global__ void finalize_metrics_kernel(double *metrics, double inv_count) { metrics[0] = metrics[1] * inv_count; }

cudaError_t finalize_metrics(double *metrics, double inv_count, cudaStream_t st) {
    finalize_metrics_kernel<<<1, 1, 0, st>>>(metrics, inv_count);
    return cudaGetLastError();
}

// tw[m] = exp(-j 2 pi m / N), from sincospi in double precision, rounded once.
__global__ void twiddle_kernel(int N, c32 *tw) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double s, c;
    sincospi(-2.0 * (double)m / (double)N, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
}

cudaError_t twiddles(int N, c32 *tw, cudaStream_t st) {
    twiddle_kernel<<<(N + 255) / 256, 256, 0, st>>>(N, tw);
    return cudaGetLastError();
}

}  // namespace fdk

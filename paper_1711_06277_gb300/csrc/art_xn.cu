// art_xn.cu -- neutral-fraction update (Sec. 2.3, Eqs. e:xn2 and e:xn3) and the substep
// size of Eq. e:dtss, elementwise over cells.
#include <cfloat>
#include <cmath>
#include <mutex>

#include "art.h"

namespace {

// Eq. e:xn3: the electron density is held at n_H (1 - x0) over dt, which makes Eq. e:xn
// linear; the solution relaxes to x_eq0 = a/(Gamma + a), a = alpha n_e, on t = 1/(Gamma + a).
__device__ __forceinline__ float xn_b(float x0, float gam, float nH, float alpha, float dt)
{
    const float a = alpha * nH * (1.f - x0);
    const float rate = gam + a;
    if (!(rate > 0.f)) return x0;
    const float xeq = a / rate;
    return xeq + (x0 - xeq) * __expf(-dt * rate);
}

// Eq. e:xn2: exact solution of the quadratic rate equation; for Gamma = 0 the closed form
// of the shielded cell.
__device__ __forceinline__ float xn_a(float x0, float gam, float nH, float alpha, float dt)
{
    const double a = (double)alpha * nH;
    if (!(gam > 0.f)) {
        const double q = (1.0 - x0) * a * dt;
        return (float)((x0 + q) / (1.0 + q));
    }
    const double g = gam;
    const double xeq = 2.0 * a / (g + 2.0 * a + sqrt(g * g + 4.0 * a * g));
    const double xp = 1.0 / xeq;
    const double K = exp(-(xp - xeq) * dt * a);
    return (float)(xeq + (xp - xeq) * (x0 - xeq) * K / ((xp - x0) + (x0 - xeq) * K));
}

__global__ void k_xn_update(long long ncell, const float* __restrict__ gamma,
                            const float* __restrict__ nH, float* __restrict__ xn,
                            float* __restrict__ nH0, float alpha, float dt, int method)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (; i < ncell; i += step) {
        const float n = nH[i];
        const float x0 = xn[i];
        const float g = gamma[i];
        float x = method == 0 ? xn_b(x0, g, n, alpha, dt) : xn_a(x0, g, n, alpha, dt);
        x = fminf(fmaxf(x, 0.f), 1.f);
        xn[i] = x;
        if (nH0) nH0[i] = x * n;
    }
}

// Per-block minimum of n_H / |I - R| (I = x n_H Gamma, R = alpha (n_H (1 - x))^2).
__global__ void k_dt_partial(long long ncell, const float* __restrict__ gamma,
                             const float* __restrict__ nH, const float* __restrict__ xn,
                             float alpha, float* __restrict__ part)
{
    __shared__ float s_min[32];
    float m = INFINITY;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (; i < ncell; i += step) {
        const float n = nH[i], x = xn[i];
        const float ne = n * (1.f - x);
        const float d = fabsf(x * n * gamma[i] - alpha * ne * ne);
        if (d > 0.f) m = fminf(m, n / d);
    }
    for (int off = 16; off > 0; off >>= 1) m = fminf(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x + 31) / 32 ? s_min[threadIdx.x] : INFINITY;
        for (int off = 16; off > 0; off >>= 1) m = fminf(m, __shfl_down_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) part[blockIdx.x] = m;
    }
}

__global__ void k_dt_final(int nparts, const float* __restrict__ part, double C, double* out)
{
    __shared__ float s_min[32];
    float m = INFINITY;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) m = fminf(m, part[i]);
    for (int off = 16; off > 0; off >>= 1) m = fminf(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x + 31) / 32 ? s_min[threadIdx.x] : INFINITY;
        for (int off = 16; off > 0; off >>= 1) m = fminf(m, __shfl_down_sync(0xffffffffu, m, off));
        if (threadIdx.x == 0) *out = isinf(m) ? (double)INFINITY : C * (double)m;
    }
}

constexpr int kDtBlocks = 1024;

}  // namespace

// ---------------------------------------------------------------------------------------
// Allocation-free variant of art_dt_substep (no counterpart in the paper).
//
// Some callers cannot call cudaMalloc: code embedded in a host framework that owns all of
// the device memory through its own pool, where a fresh allocation fails or fragments that
// pool, and latency-critical loops that cannot afford the implicit device synchronization of
// cudaMalloc/cudaFree. For them the per-block partial minima live in this fixed array,
// which every GPU that loads the library keeps for the life of the process: one float per
// 256-cell tile, so inputs of up to ART_DT_STATIC_MAX_CELLS cells.
// ---------------------------------------------------------------------------------------
namespace {

constexpr int kStaticTiles = 65536;  // ART_DT_STATIC_MAX_CELLS / 256
static __device__ __align__(256) float g_dt_partials[kStaticTiles];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float* g_static_ptr[kMaxDevices] = {};

// Device address of g_dt_partials on the current device, looked up once per device. In
// host code the symbol's name is only a host-side stand-in and must never reach a kernel.
int static_partials(float** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ART_ECUDA;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dt_partials) != cudaSuccess || !p) return ART_ECUDA;
        g_static_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_static_ptr[dev];
    return ART_OK;
}

}  // namespace

extern "C" {

int art_xn_update(void* stream, long long ncell, const float* d_gamma, const float* d_nH,
                  float* d_xn, float* d_nH0, double alpha_B, double dt, int method)
{
    if (ncell < 0 || (ncell > 0 && (!d_gamma || !d_nH || !d_xn))) return ART_EINVAL;
    if (!(alpha_B > 0.0) || !(dt >= 0.0) || !std::isfinite(dt) || (method != 0 && method != 1))
        return ART_EINVAL;
    if (ncell == 0) return ART_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ART_ECUDA;
    // a grid-stride loop over 16 resident blocks of 256 threads per SM
    const long long cap = 16ll * (sms > 0 ? sms : 1);
    const int blocks = (int)((ncell + 255) / 256 < cap ? (ncell + 255) / 256 : cap);
    k_xn_update<<<blocks, 256, 0, (cudaStream_t)stream>>>(ncell, d_gamma, d_nH, d_xn, d_nH0,
                                                          (float)alpha_B, (float)dt, method);
    return cudaGetLastError() == cudaSuccess ? ART_OK : ART_ECUDA;
}

long long art_dt_scratch_bytes(long long ncell)
{
    (void)ncell;
    return (long long)kDtBlocks * (long long)sizeof(float);
}

int art_dt_substep(void* stream, long long ncell, const float* d_gamma, const float* d_nH,
                   const float* d_xn, double alpha_B, double C, void* d_scratch, double* d_dt)
{
    if (ncell <= 0 || !d_gamma || !d_nH || !d_xn || !d_scratch || !d_dt) return ART_EINVAL;
    if (!(alpha_B > 0.0) || !(C > 0.0)) return ART_EINVAL;
    long long want = (ncell + 255) / 256;
    const int blocks = (int)(want < kDtBlocks ? want : kDtBlocks);
    cudaStream_t s = (cudaStream_t)stream;
    k_dt_partial<<<blocks, 256, 0, s>>>(ncell, d_gamma, d_nH, d_xn, (float)alpha_B,
                                        (float*)d_scratch);
    k_dt_final<<<1, 1024, 0, s>>>(blocks, (const float*)d_scratch, C, d_dt);
    return cudaGetLastError() == cudaSuccess ? ART_OK : ART_ECUDA;
}

int art_dt_substep_static(void* stream, long long ncell, const float* d_gamma, const float* d_nH,
                          const float* d_xn, double alpha_B, double C, double* d_dt)
{
    if (ncell <= 0 || !d_gamma || !d_nH || !d_xn || !d_dt) return ART_EINVAL;
    if (ncell > ART_DT_STATIC_MAX_CELLS) return ART_EINVAL;  // beyond the fixed scratch
    if (!(alpha_B > 0.0) || !(C > 0.0)) return ART_EINVAL;
    float* partials = nullptr;
    const int rc = static_partials(&partials);
    if (rc != ART_OK) return rc;
    // one tile of 256 cells per block: every partial read below is written first by its
    // block in this call, so nothing carries over from an earlier call
    const int tiles = (int)((ncell + 255) / 256);
    cudaStream_t s = (cudaStream_t)stream;
    k_dt_partial<<<tiles, 256, 0, s>>>(ncell, d_gamma, d_nH, d_xn, (float)alpha_B, partials);
    k_dt_final<<<1, 1024, 0, s>>>(tiles, partials, C, d_dt);
    return cudaGetLastError() == cudaSuccess ? ART_OK : ART_ECUDA;
}

}  // extern "C"

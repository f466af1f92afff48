// Heterogeneous density of the transformed CSD equation [Sec. 2, Eq. BoltzmannCSDTrafo] and its
// dose [Sec. 2, dose definition].
//
// After the energy transform the equation reads d_t psi + Omega . grad(psi / rho) + Sigma_t(t) psi
// = scattering, with rho the tissue density and t the transformed energy (pseudo-time): the flux
// transports psi / rho (the kernels of flux.cu scale each row by its cell's 1/rho) and the cross
// sections depend on t only (the caller passes this step's values as the per-cell sigma arrays).
// kitrt_mn_set_density stores 1/rho in the solver; kitrt_dose_accumulate adds one pseudo-time
// step's dose: with psi~ = S_w rho psi and dE = S_w dE~, the dose D = 1/rho int S psi dOmega dE
// becomes 1/rho int Phi~ S_w dE~ with Phi~ = int psi~ dOmega = u_0 / m_0.
#include <math.h>

#include "kitrt_internal.cuh"

namespace {

// 1/rho in FP64 and FP32; counts entries that are not positive and finite.
__global__ void invrho_kernel(const double *__restrict__ rho, double *__restrict__ inv,
                              float *__restrict__ inv32, int C, unsigned long long *__restrict__ bad)
{
    unsigned nbad = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
        const double r = rho[i];
        const bool ok = r > 0.0 && isfinite(r);
        nbad += ok ? 0u : 1u;
        const double v = ok ? 1.0 / r : 1.0;
        inv[i] = v;
        inv32[i] = (float)v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(bad, (unsigned long long)nbad);
}

__global__ void dose_kernel(const double *__restrict__ u, const double *__restrict__ invrho, int n,
                            double scale, double *__restrict__ dose, int C)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C; i += gridDim.x * blockDim.x) {
        const double r = invrho ? invrho[i] : 1.0;
        dose[i] += scale * u[(size_t)i * n] * r;
    }
}

int grid_of(const kitrt_mn *mn, int C)
{
    int blocks = (C + 255) / 256;
    if (blocks > mn->nsm * 8) blocks = mn->nsm * 8;
    return blocks > 0 ? blocks : 1;
}

}  // namespace

extern "C" int32_t kitrt_mn_set_density(kitrt_mn *mn, const double *rho, void *stream)
{
    if (!mn) return KITRT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (!rho) {
        mn->d_invrho = nullptr;
        mn->d_invrho32 = nullptr;
        return KITRT_OK;
    }
    const int C = mn->mesh->C;
    if (!mn->d_rho_store) {
        // 1/rho (FP64) then 1/rho (FP32) in one allocation, made once per solver and kept (the
        // solver's workspace; freed by kitrt_mn_destroy)
        void *p = nullptr;
        if (cudaMalloc(&p, (size_t)C * (sizeof(double) + sizeof(float)) + 256) != cudaSuccess)
            return KITRT_ENOMEM;
        mn->allocs.push_back(p);
        mn->d_rho_store = static_cast<double *>(p);
    }
    double *inv = mn->d_rho_store;
    float *inv32 = reinterpret_cast<float *>(inv + C);
    if (cudaMemsetAsync(mn->d_check, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess)
        return KITRT_ECUDA;
    {
        LaunchScope ls(mn, PK_OTHER, s, C);
        invrho_kernel<<<grid_of(mn, C), 256, 0, s>>>(rho, inv, inv32, C, mn->d_check);
    }
    if (cudaGetLastError() != cudaSuccess) return KITRT_ECUDA;
    if (cudaMemcpyAsync(mn->h_check, mn->d_check, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return KITRT_ECUDA;
    if (mn->h_check[0] != 0) {
        // a rejected density leaves the solver without one (the copy above overwrote the old)
        mn->d_invrho = nullptr;
        mn->d_invrho32 = nullptr;
        return KITRT_EINVAL;
    }
    mn->d_invrho = inv;
    mn->d_invrho32 = inv32;
    return KITRT_OK;
}

extern "C" int32_t kitrt_dose_accumulate(kitrt_mn *mn, const double *u, double S, double dt,
                                         double *dose, void *stream)
{
    if (!mn || !u || !dose || !isfinite(S) || !isfinite(dt)) return KITRT_EINVAL;
    const int C = mn->mesh->C;
    cudaStream_t s = (cudaStream_t)stream;
    // dt S u_0 / (m_0 rho) with 1 / m_0 = sqrt(4 pi)
    const double scale = dt * S * sqrt(4.0 * 3.14159265358979323846);
    {
        LaunchScope ls(mn, PK_OTHER, s, C);
        dose_kernel<<<grid_of(mn, C), 256, 0, s>>>(u, mn->d_invrho, mn->n, scale, dose, C);
    }
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

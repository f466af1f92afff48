// Small multilayer perceptron of the learned entropy closure: y = W4 s(W3 s(W2 s(W1 x + b1) + b2)
// + b3) + b4 with s = softplus, trained in FP32 with the library's own kernels (tiled SIMT GEMMs
// with split-K, elementwise softplus and its derivative sigmoid, column sums, mean-squared loss,
// Adam), and evaluated inside the learned M_N step with BF16-rounded weights and activations and
// FP32 accumulation.
//
// The paper closes the M_N system with input-convex networks trained elsewhere [Sec. 3.1, neural
// entropy closures; Sec. 7.2 M_1 neural closure]; this library trains its own plain MLP on
// (normalised moments, alpha) pairs produced by its Newton closure.
//
// Parameter packing (FP32, row-major [in x out]): W1[din*H] b1[H] W2[H*H] b2[H] W3[H*H] b3[H]
// W4[H*dout] b4[dout]. Loss = 1/(2B) sum_b ||y_b - t_b||^2.
#include <cuda_bf16.h>
#include <math.h>

#include "kitrt_internal.cuh"

namespace {

constexpr int kTile = 64, kTK = 16;

// C[M x N] (+)= A[M x K] B[K x N] with element (i, k) of A at A[i * as0 + k * as1] and (k, j) of
// B at B[k * bs0 + j * bs1] (so transposes are strides). Optional bias per column; with
// gridDim.z > 1 the K range is split and partial products are added atomically (C zeroed first).
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, const float *__restrict__ A, int as0, int as1,
            const float *__restrict__ B, int bs0, int bs1, float *__restrict__ Cm, int ldc,
            const float *__restrict__ bias, int accumulate)
{
    __shared__ float sA[kTK][kTile + 1];
    __shared__ float sB[kTK][kTile + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row0 = blockIdx.y * kTile, col0 = blockIdx.x * kTile;
    const int kper = (K + gridDim.z - 1) / gridDim.z;
    const int kbeg = blockIdx.z * kper, kend = min(K, kbeg + kper);
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += kTK) {
        for (int idx = threadIdx.x; idx < kTK * kTile; idx += 256) {
            const int kk = idx / kTile, mm = idx % kTile;
            const int gk = k0 + kk;
            sA[kk][mm] = (gk < kend && row0 + mm < M) ? A[(size_t)(row0 + mm) * as0 + (size_t)gk * as1] : 0.0f;
            sB[kk][mm] = (gk < kend && col0 + mm < N) ? B[(size_t)gk * bs0 + (size_t)(col0 + mm) * bs1] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sA[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = sB[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = row0 + ty * 4 + i, c = col0 + tx * 4 + j;
            if (r >= M || c >= N) continue;
            float v = acc[i][j];
            if (bias && blockIdx.z == 0) v += bias[c];
            if (gridDim.z > 1 || accumulate) atomicAdd(&Cm[(size_t)r * ldc + c], v);
            else Cm[(size_t)r * ldc + c] = v;
        }
}

__device__ __forceinline__ float softplus_f(float x) { return x > 0.0f ? x + log1pf(expf(-x)) : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.0f / (1.0f + expf(-x)); }

__global__ void softplus_kernel(const float *__restrict__ Z, float *__restrict__ Hh, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        Hh[i] = softplus_f(Z[i]);
}

// dZ = dH * sigmoid(Z)
__global__ void dsoftplus_kernel(const float *__restrict__ Z, const float *__restrict__ dH, float *__restrict__ dZ,
                                 size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dZ[i] = dH[i] * sigmoid_f(Z[i]);
}

// dY = (Y - T) / B and the loss 1/(2B) sum (Y - T)^2 (atomically into *loss, zeroed first).
__global__ void mse_kernel(const float *__restrict__ Y, const float *__restrict__ Tt, float *__restrict__ dY,
                           float *__restrict__ loss, int B, int dout)
{
    float part = 0.0f;
    const size_t n = (size_t)B * dout;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float r = Y[i] - Tt[i];
        dY[i] = r / B;
        part += 0.5f * r * r / B;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// g[j] = sum_r D[r, j] (column sums, atomically accumulated; g zeroed first)
__global__ void colsum_kernel(const float *__restrict__ Dm, float *__restrict__ g, int R, int Ncol)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Ncol) return;
    const int per = (R + gridDim.y - 1) / gridDim.y;
    const int r0 = blockIdx.y * per, r1 = min(R, r0 + per);
    float s = 0.0f;
    for (int r = r0; r < r1; ++r) s += Dm[(size_t)r * Ncol + j];
    atomicAdd(&g[j], s);
}

__global__ void adam_kernel(int P, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
        const float mk = b1 * m[k] + (1.0f - b1) * g[k];
        const float vk = b2 * v[k] + (1.0f - b2) * g[k] * g[k];
        m[k] = mk;
        v[k] = vk;
        p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    }
}

struct Lay {
    const float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
};

Lay unpack(const float *p, int din, int H, int dout)
{
    Lay L;
    L.W1 = p;
    L.b1 = L.W1 + din * H;
    L.W2 = L.b1 + H;
    L.b2 = L.W2 + H * H;
    L.W3 = L.b2 + H;
    L.b3 = L.W3 + H * H;
    L.W4 = L.b3 + H;
    L.b4 = L.W4 + H * dout;
    return L;
}

// C = X W (+ b): X [B x K] row-major, W [K x N] row-major
int gemm_xw(int B, int K, int N, const float *X, const float *W, const float *b, float *C, cudaStream_t s)
{
    dim3 grid((N + kTile - 1) / kTile, (B + kTile - 1) / kTile, 1);
    gemm_kernel<<<grid, 256, 0, s>>>(B, N, K, X, K, 1, W, N, 1, C, N, b, 0);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

// dX = dY W^T: dY [B x N], W [K x N] -> dX [B x K]
int gemm_dyWt(int B, int K, int N, const float *dY, const float *W, float *dX, cudaStream_t s)
{
    dim3 grid((K + kTile - 1) / kTile, (B + kTile - 1) / kTile, 1);
    gemm_kernel<<<grid, 256, 0, s>>>(B, K, N, dY, N, 1, W, 1, N, dX, K, nullptr, 0);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

// gW = X^T dY: X [B x K], dY [B x N] -> gW [K x N], split over the batch (gW zeroed first)
int gemm_xtdy(int B, int K, int N, const float *X, const float *dY, float *gW, cudaStream_t s)
{
    int splits = (B + 255) / 256;
    if (splits > 64) splits = 64;
    dim3 grid((N + kTile - 1) / kTile, (K + kTile - 1) / kTile, splits > 0 ? splits : 1);
    gemm_kernel<<<grid, 256, 0, s>>>(K, N, B, X, 1, K, dY, N, 1, gW, N, nullptr, 1);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int blocks_for(size_t n) { return (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096); }

}  // namespace

extern "C" {

int32_t kitrt_mlp_param_count(int32_t din, int32_t H, int32_t dout)
{
    return din * H + H + 2 * (H * H + H) + H * dout + dout;
}

int32_t kitrt_mlp_work_floats(int32_t B, int32_t H, int32_t dout) { return B * (8 * H + 2 * dout); }

int32_t kitrt_mlp_forward(int32_t din, int32_t H, int32_t dout, const float *params, const float *X,
                          float *Y, int32_t B, float *work, void *stream)
{
    if (din < 1 || H < 1 || dout < 1 || B < 0 || !params || !X || !Y || !work) return KITRT_EINVAL;
    if (B == 0) return KITRT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const Lay L = unpack(params, din, H, dout);
    float *Z = work, *Ha = work + (size_t)B * H, *Hb = work + 2 * (size_t)B * H;
    const size_t BH = (size_t)B * H;
    int rc = gemm_xw(B, din, H, X, L.W1, L.b1, Z, s);
    softplus_kernel<<<blocks_for(BH), 256, 0, s>>>(Z, Ha, BH);
    rc = rc ? rc : gemm_xw(B, H, H, Ha, L.W2, L.b2, Z, s);
    softplus_kernel<<<blocks_for(BH), 256, 0, s>>>(Z, Hb, BH);
    rc = rc ? rc : gemm_xw(B, H, H, Hb, L.W3, L.b3, Z, s);
    softplus_kernel<<<blocks_for(BH), 256, 0, s>>>(Z, Ha, BH);
    rc = rc ? rc : gemm_xw(B, H, dout, Ha, L.W4, L.b4, Y, s);
    if (rc) return rc;
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int32_t kitrt_mlp_loss_grad(int32_t din, int32_t H, int32_t dout, const float *params, const float *X,
                            const float *Tt, int32_t B, float *grad, float *loss, float *work, void *stream)
{
    if (din < 1 || H < 1 || dout < 1 || B < 1 || !params || !X || !Tt || !grad || !loss || !work)
        return KITRT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const Lay L = unpack(params, din, H, dout);
    const size_t BH = (size_t)B * H;
    float *Z1 = work, *H1 = Z1 + BH, *Z2 = H1 + BH, *H2 = Z2 + BH, *Z3 = H2 + BH, *H3 = Z3 + BH;
    float *dH = H3 + BH, *dZ = dH + BH, *Y = dZ + BH, *dY = Y + (size_t)B * dout;
    const int P = kitrt_mlp_param_count(din, H, dout);
    float *gW1 = grad, *gb1 = gW1 + din * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H,
          *gb3 = gW3 + H * H, *gW4 = gb3 + H, *gb4 = gW4 + H * dout;
    if (cudaMemsetAsync(grad, 0, sizeof(float) * P, s) != cudaSuccess) return KITRT_ECUDA;
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return KITRT_ECUDA;
    int rc = gemm_xw(B, din, H, X, L.W1, L.b1, Z1, s);
    softplus_kernel<<<blocks_for(BH), 256, 0, s>>>(Z1, H1, BH);
    rc = rc ? rc : gemm_xw(B, H, H, H1, L.W2, L.b2, Z2, s);
    softplus_kernel<<<blocks_for(BH), 256, 0, s>>>(Z2, H2, BH);
    rc = rc ? rc : gemm_xw(B, H, H, H2, L.W3, L.b3, Z3, s);
    softplus_kernel<<<blocks_for(BH), 256, 0, s>>>(Z3, H3, BH);
    rc = rc ? rc : gemm_xw(B, H, dout, H3, L.W4, L.b4, Y, s);
    mse_kernel<<<blocks_for((size_t)B * dout), 256, 0, s>>>(Y, Tt, dY, loss, B, dout);
    // layer 4
    rc = rc ? rc : gemm_xtdy(B, H, dout, H3, dY, gW4, s);
    dim3 cg4((dout + 255) / 256, 32);
    colsum_kernel<<<cg4, 256, 0, s>>>(dY, gb4, B, dout);
    rc = rc ? rc : gemm_dyWt(B, H, dout, dY, L.W4, dH, s);
    // layers 3, 2, 1
    const float *Zs[3] = {Z3, Z2, Z1};
    const float *ins[3] = {H2, H1, X};
    const float *Ws[3] = {L.W3, L.W2, L.W1};
    float *gWs[3] = {gW3, gW2, gW1}, *gbs[3] = {gb3, gb2, gb1};
    const int dins[3] = {H, H, din};
    for (int l = 0; l < 3 && !rc; ++l) {
        dsoftplus_kernel<<<blocks_for(BH), 256, 0, s>>>(Zs[l], dH, dZ, BH);
        rc = gemm_xtdy(B, dins[l], H, ins[l], dZ, gWs[l], s);
        dim3 cg((H + 255) / 256, 32);
        colsum_kernel<<<cg, 256, 0, s>>>(dZ, gbs[l], B, H);
        if (l < 2 && !rc) rc = gemm_dyWt(B, H, H, dZ, Ws[l], dH, s);
    }
    if (rc) return rc;
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

int32_t kitrt_mlp_adam(int32_t P, float *params, const float *grad, float *m, float *v, int32_t t, float lr,
                       float b1, float b2, float eps, void *stream)
{
    if (P < 1 || t < 1 || !params || !grad || !m || !v) return KITRT_EINVAL;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    adam_kernel<<<blocks_for(P), 256, 0, (cudaStream_t)stream>>>(P, params, grad, m, v, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Inference inside the learned step: one thread per listed cell. Features v = u_{1..n-1}/u_0,
// standardised; the network in BF16 weights and BF16-rounded activations with FP32 accumulation;
// the output de-standardised to alpha_{1..n-1}, written in FP64 to the Newton state (alpha_0 is
// fixed by the exact mass constraint afterwards).
// ---------------------------------------------------------------------------------------------
namespace {

constexpr int kH = 64;

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Dense layer for one thread's sample: out[j] = act(b[j] + sum_i in[i] W[i][j]) with in/out
// activations in shared memory laid out [unit][thread] (conflict-free), outputs produced 16 at a
// time to bound registers.
template <int DIN, int DOUT, bool ACT>
__device__ __forceinline__ void dense(const float *__restrict__ W, const float *__restrict__ b,
                                      const float *in, float *out, int tid, int nthr)
{
#pragma unroll
    for (int j0 = 0; j0 < DOUT; j0 += 16) {
        float acc[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) acc[jj] = (j0 + jj < DOUT) ? b[j0 + jj] : 0.0f;
#pragma unroll 4
        for (int i = 0; i < DIN; ++i) {
            const float x = in[i * nthr + tid];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj)
                if (j0 + jj < DOUT) acc[jj] = fmaf(x, W[i * DOUT + j0 + jj], acc[jj]);
        }
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
            if (j0 + jj < DOUT) out[(j0 + jj) * nthr + tid] = ACT ? bf(softplus_f(acc[jj])) : acc[jj];
    }
}

template <int DIO>
__global__ void __launch_bounds__(128)
mlp_infer_kernel(const __nv_bfloat16 *__restrict__ wq, const float *__restrict__ norm, const double *__restrict__ u,
                 const int32_t *__restrict__ list, const int32_t *__restrict__ cnt_ptr, int C, double *__restrict__ alpha)
{
    // weights as floats in shared memory (values already rounded to BF16), then two activation
    // buffers of [64 units x 128 threads]
    constexpr int P = DIO * kH + kH + 2 * (kH * kH + kH) + kH * DIO + DIO;
    constexpr int nthr = 128;
    extern __shared__ float sw[];
    float *bufA = sw + ((P + 31) / 32) * 32, *bufB = bufA + kH * nthr;
    const int count = list ? *cnt_ptr : C;
    // the grid is sized for every cell; blocks past the listed samples leave at once (uniform)
    if ((int)(blockIdx.x * nthr) >= count) return;
    for (int k = threadIdx.x; k < P; k += blockDim.x) sw[k] = __bfloat162float(wq[k]);
    __syncthreads();
    const float *W1 = sw, *b1 = W1 + DIO * kH, *W2 = b1 + kH, *b2 = W2 + kH * kH, *W3 = b2 + kH, *b3 = W3 + kH * kH,
                *W4 = b3 + kH, *b4 = W4 + kH * DIO;
    const float *xm = norm, *xs = norm + DIO, *ym = norm + 2 * DIO, *ys = norm + 3 * DIO;
    constexpr int n = DIO + 1;
    const int tid = threadIdx.x;
    // uniform trip count per block so that every thread reaches the same barriers
    const int rounds = (count + gridDim.x * nthr - 1) / (gridDim.x * nthr);
    for (int rd = 0; rd < rounds; ++rd) {
        const int it = (rd * gridDim.x + blockIdx.x) * nthr + tid;
        const bool live = it < count;
        const int cell = live ? (list ? list[it] : it) : 0;
        if (live) {
            const double u0 = u[(size_t)cell * n];
            for (int i = 0; i < DIO; ++i)
                bufB[i * nthr + tid] = bf(((float)(u[(size_t)cell * n + 1 + i] / u0) - xm[i]) / xs[i]);
        }
        dense<DIO, kH, true>(W1, b1, bufB, bufA, tid, nthr);
        dense<kH, kH, true>(W2, b2, bufA, bufB, tid, nthr);
        dense<kH, kH, true>(W3, b3, bufB, bufA, tid, nthr);
        dense<kH, DIO, false>(W4, b4, bufA, bufB, tid, nthr);
        if (live)
            for (int j = 0; j < DIO; ++j)
                alpha[(size_t)cell * n + 1 + j] = (double)(bufB[j * nthr + tid] * ys[j] + ym[j]);
    }
}

}  // namespace

int launch_mlp_infer(kitrt_mn *mn, const double *u, const int32_t *list, const int32_t *cnt, int C,
                     double *alpha, cudaStream_t s)
{
    const int dio = mn->n - 1;
    const int P = kitrt_mlp_param_count(dio, kH, dio);
    const size_t smem = sizeof(float) * (((P + 31) / 32) * 32 + 2 * kH * 128);
    int blocks = (C + 127) / 128;
    if (blocks > mn->nsm * 8) blocks = mn->nsm * 8;
    if (blocks < 1) blocks = 1;
    LaunchScope ls(mn, PK_MLP, s, C);
#define INFER_CASE(D)                                                                                        \
    case D:                                                                                                  \
        if (ensure_dyn_smem(mlp_infer_kernel<D>, smem)) return KITRT_ECUDA;                                 \
        mlp_infer_kernel<D><<<blocks, 128, smem, s>>>((const __nv_bfloat16 *)mn->d_mlp16, mn->d_mlp_norm, u, list, \
                                                      cnt, C, alpha);                                        \
        break;
    switch (dio) {
        INFER_CASE(2)
        INFER_CASE(5)
        INFER_CASE(9)
        INFER_CASE(14)
        INFER_CASE(20)
    default: return KITRT_EINVAL;
    }
#undef INFER_CASE
    return cudaGetLastError() == cudaSuccess ? KITRT_OK : KITRT_ECUDA;
}

// lsd_mlp.cu -- per-atom energy MLP and its input gradient, FP32 on the CUDA
// cores: h_l = W_l a_{l-1} + b_l, a_l = SiLU(h_l), y = w_out.a_L + b_out,
// e = head(y); backward g_L = e'(y) w_out * SiLU'(h_L),
// g_{l-1} = (W_l^T g_l) * SiLU'(h_{l-1}), dE/dx = W_1^T g_1.
//
// One CTA owns a tile of 32 rows for the whole forward and backward pass:
// activations and SiLU' stay in shared memory, weights stream through a
// double-buffered shared-memory stage.
// 256 threads = 8 row groups of 4 rows x 32 lanes over columns (strided by 32),
// so activation reads are warp broadcasts and weight reads are coalesced.
#include "lsd_common.cuh"
#include "lsd_kernels.h"

namespace lsd {

constexpr int kTM = 32;

constexpr int kStageFloats = 4096;   // one staged weight chunk (16 KB); two are in flight

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// acc[4][RN] = A[32 x KD] (shared, row stride lda) x B[KD x 32*RN] (global, row-major).
// B streams through two shared buffers of KC rows: the copy of chunk c+1
// (cp.async, 16 B per thread-request) is in flight while chunk c is consumed.
template <int RN>
__device__ __forceinline__ void gemm_rows4(const float *__restrict__ A, int lda, int KD, const float *__restrict__ B,
                                           float *__restrict__ Bs, float (&acc)[4][8]) {
    constexpr int NC = 32 * RN;
    constexpr int KC = kStageFloats / NC >= 32 ? 32 : kStageFloats / NC;   // 32 rows, 16 for NC = 256
    const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
    const float *a0 = A + (rg * 4) * lda;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
    const int nch = KD / KC;
    auto issue = [&](int ch) {
        const float *src = B + (size_t)ch * KC * NC;
        float *dst = Bs + (ch & 1) * kStageFloats;
        for (int t = threadIdx.x; t < KC * NC / 4; t += blockDim.x) cp_async16(dst + 4 * t, src + 4 * t);
        cp_async_commit();
    };
    issue(0);
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) {
            issue(ch + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float *bs = Bs + (ch & 1) * kStageFloats;
        const int k0 = ch * KC;
#pragma unroll 4
        for (int k = 0; k < KC; ++k) {
            float a[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = a0[r * lda + k0 + k];
            float b[RN];
#pragma unroll
            for (int c = 0; c < RN; ++c) b[c] = bs[k * NC + lane + 32 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < RN; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();   // the buffer is refilled two chunks later
    }
}

__device__ __forceinline__ void gemm_dispatch(int ncols, const float *A, int lda, int KD, const float *B, float *Bs,
                                              float (&acc)[4][8]) {
    switch (ncols >> 5) {
        case 1: gemm_rows4<1>(A, lda, KD, B, Bs, acc); break;
        case 2: gemm_rows4<2>(A, lda, KD, B, Bs, acc); break;
        case 3: gemm_rows4<3>(A, lda, KD, B, Bs, acc); break;
        case 4: gemm_rows4<4>(A, lda, KD, B, Bs, acc); break;
        case 5: gemm_rows4<5>(A, lda, KD, B, Bs, acc); break;
        case 6: gemm_rows4<6>(A, lda, KD, B, Bs, acc); break;
        case 7: gemm_rows4<7>(A, lda, KD, B, Bs, acc); break;
        default: gemm_rows4<8>(A, lda, KD, B, Bs, acc); break;
    }
}

__global__ void __launch_bounds__(256) mlp_fp32_kernel(const float *__restrict__ X, int M, PotDev P,
                                                       float *__restrict__ E_mlp, float *__restrict__ dEdX) {
    pdl_wait();
    pdl_release();
    extern __shared__ float sm[];
    const int d0p = P.d0p, W = P.width, L = P.n_layers;
    const int ld = d0p > W ? d0p : W;
    float *buf0 = sm;
    float *buf1 = buf0 + kTM * ld;
    float *spr = buf1 + kTM * ld;                   // [L][kTM][W] SiLU'(h)
    float *sdedy = spr + (size_t)L * kTM * W;       // [kTM]
    float *Bs = sdedy + kTM;                        // 2 x kStageFloats staged weight chunks
    const int tid = threadIdx.x, lane = tid & 31, rg = tid >> 5;
    const int row0 = blockIdx.x * kTM;

    for (int idx = tid; idx < kTM * d0p; idx += blockDim.x) {
        const int r = idx / d0p, f = idx - r * d0p;
        buf0[r * ld + f] = (row0 + r < M) ? X[(size_t)(row0 + r) * d0p + f] : 0.f;
    }
    __syncthreads();
    float *in = buf0, *out = buf1;
    int din = d0p;
    float acc[4][8];
    for (int l = 0; l < L; ++l) {
        gemm_dispatch(W, in, ld, din, P.Wt[l], Bs, acc);
        const int RN = W >> 5;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < RN; ++c) {
                const int row = rg * 4 + r, col = lane + 32 * c;
                const float h = acc[r][c] + P.b[l][col];
                out[row * ld + col] = siluf_(h);
                spr[((size_t)l * kTM + row) * W + col] = dsiluf_(h);
            }
        __syncthreads();
        float *t = in; in = out; out = t;
        din = W;
    }
    // y = w_out . a_L + b_out, per row (warp rg owns rows 4rg..4rg+3)
    for (int r = 0; r < 4; ++r) {
        const int row = rg * 4 + r;
        float s = 0.f;
        for (int col = lane; col < W; col += 32) s += in[row * ld + col] * P.wout[col];
        s = warp_sum(s);
        if (lane == 0) {
            const float y = s + P.bout;
            float e, dedy;
            if (P.head == 1) { e = y; dedy = 1.f; }
            else {
                const float t = tanhf(y);
                e = P.head_scale * t;
                dedy = P.head_scale * (1.f - t * t);
            }
            sdedy[row] = dedy;
            if (row0 + row < M) E_mlp[row0 + row] = e;
        }
    }
    __syncthreads();
    // g_L = e'(y) w_out * SiLU'(h_L)
    for (int idx = tid; idx < kTM * W; idx += blockDim.x) {
        const int r = idx / W, c = idx - r * W;
        out[r * ld + c] = sdedy[r] * P.wout[c] * spr[((size_t)(L - 1) * kTM + r) * W + c];
    }
    __syncthreads();
    { float *t = in; in = out; out = t; }
    for (int l = L - 1; l >= 0; --l) {
        const int dout = (l == 0) ? d0p : W;
        gemm_dispatch(dout, in, ld, W, P.Wn[l], Bs, acc);
        const int RN = dout >> 5;
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < RN; ++c) {
                const int row = rg * 4 + r, col = lane + 32 * c;
                if (l > 0) out[row * ld + col] = acc[r][c] * spr[((size_t)(l - 1) * kTM + row) * W + col];
                else if (row0 + row < M) dEdX[(size_t)(row0 + row) * d0p + col] = acc[r][c];
            }
        __syncthreads();
        float *t = in; in = out; out = t;
    }
}

size_t mlp_fp32_smem_bytes(const PotDev &P) {
    const int ld = P.d0p > P.width ? P.d0p : P.width;
    return ((size_t)2 * kTM * ld + (size_t)P.n_layers * kTM * P.width + kTM + 2 * (size_t)kStageFloats) * sizeof(float);
}

void launch_mlp_fp32(const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX, cudaStream_t s) {
    launch_dependent(mlp_fp32_kernel, (M + kTM - 1) / kTM, 256, mlp_fp32_smem_bytes(P), s, X, M, P, E_mlp, dEdX);
}

cudaError_t mlp_kernels_setup(int max_smem) {
    return cudaFuncSetAttribute(mlp_fp32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

}  // namespace lsd

// lsd_mlp_tc.cu -- the per-atom energy MLP and its input gradient on the
// 5th-generation tensor cores (tcgen05), BF16 operands, FP32 accumulation in
// tensor memory.  Same mathematics as lsd_mlp.cu:
//   forward  h_l = W_l a_{l-1} + b_l, a_l = SiLU(h_l), y = w_out.a_L + b_out
//   backward g_L = e'(y) w_out * SiLU'(h_L), g_{l-1} = (W_l^T g_l) * SiLU'(h_{l-1}),
//            dE/dx = W_1^T g_1
// Every layer is a GEMM D[128 x N] = A[128 x K] B[N x K]^T with the tile's
// 128 rows in the 128 TMEM lanes:
//   forward  A = a_{l-1} (bf16),  B = W_l   [W x din]  (N = W,   K = din)
//   backward A = g_l     (bf16),  B = W_l^T [din x W]  (N = din, K = W)
// A lives in shared memory in the 128-byte-swizzled K-major layout (panels of
// 64 bf16 per row), written by the epilogue of the previous GEMM.  B streams
// from global memory by TMA (2-D tiled copies, 128-byte swizzle) in chunks of
// 64 K-columns through two stages, synchronised with mbarriers.  One thread
// issues the TMA copies and MMAs (M = 128, K = 16 per instruction) and commits
// their completion to mbarriers; the 128 threads (one per row) run the
// epilogues from TMEM with tcgen05.ld.  SiLU'(h) of each layer is kept in a
// per-CTA global scratch slot (bf16) that stays resident in L2.
// The grid is persistent: one CTA per SM, looping over 128-row tiles.
// Every mbarrier wait gives up after about a second and records an error.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lsd.h"
#include "lsd_common.cuh"
#include "lsd_kernels.h"
#include "lsd_tc.cuh"

namespace lsd {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;
constexpr int kPanelElems = 64;                   // bf16 elements per 128-byte swizzled row
constexpr int kPanelBytes = kTcRows * 128;        // one K-panel of A: 16 KB
constexpr int kMaxPanels = 4;                     // K up to 256
constexpr int kStageBytes = 256 * 128;            // one B chunk: up to 256 rows x 128 B

struct TcSmem {
    uint32_t a;          // A operand panels
    uint32_t b0;         // B stage s at b0 + s kStageBytes
    uint32_t full0;      // TMA landed (stage s at full0 + 8 s)
    uint32_t empty0;     // MMAs done with the stage (empty0 + 8 s)
    uint32_t done;       // all MMAs of a GEMM done
    uint32_t tslot;      // TMEM base address
    __device__ __forceinline__ uint32_t b(int s) const { return b0 + (uint32_t)s * kStageBytes; }
    __device__ __forceinline__ uint32_t full(int s) const { return full0 + 8u * (uint32_t)s; }
    __device__ __forceinline__ uint32_t empty(int s) const { return empty0 + 8u * (uint32_t)s; }
};

// One GEMM: thread 0 streams the K-chunks of B by TMA and issues the MMAs;
// every thread then waits for the accumulator.  chunk counts TMA chunks over
// the whole kernel (stage = chunk & 1, use = chunk >> 1); gemm counts GEMMs.
__device__ __forceinline__ bool tc_gemm(const TcSmem &S, const CUtensorMap *map, int K, int N, uint32_t tmem,
                                        uint32_t &chunk, uint32_t &gemm) {
    bool ok = true;
    const int nk = (K + kPanelElems - 1) / kPanelElems;
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        const uint32_t idesc = tc::idesc_f32acc(tc::kFmtBF16, kTcRows, N);
        const uint32_t bytes = (uint32_t)N * 128u;
        auto issue = [&](uint32_t c, int kc) {
            const int s = c & 1;
            if (c >= 2 && ok) ok = tc::mbar_wait(S.empty(s), ((c >> 1) - 1) & 1);
            if (!ok) return;
            tc::mbar_expect_tx(S.full(s), bytes);
            tc::tma_load_2d(S.b(s), map, kc * kPanelElems, 0, S.full(s));
        };
        const uint32_t c0 = chunk;
        issue(c0, 0);
        for (int kc = 0; kc < nk && ok; ++kc) {
            const uint32_t c = c0 + kc;
            if (kc + 1 < nk) issue(c + 1, kc + 1);
            const int s = c & 1;
            if (!tc::mbar_wait(S.full(s), (c >> 1) & 1)) { ok = false; break; }
            tc::fence_after_sync();
            const int kend = min(kPanelElems, K - kc * kPanelElems);
            for (int k16 = 0; k16 < kend; k16 += 16) {
                const uint64_t ad = tc::sdesc_sw128(S.a + kc * kPanelBytes + k16 * 2);
                const uint64_t bd = tc::sdesc_sw128(S.b(s) + k16 * 2);
                tc::mma_f16(tmem, ad, bd, idesc, (kc | k16) != 0);
            }
            tc::mma_commit(S.empty(s));
        }
        tc::mma_commit(S.done);
    }
    chunk += nk;
    // everyone waits for the accumulator of this GEMM
    if (!tc::mbar_wait(S.done, gemm & 1)) ok = false;
    ++gemm;
    tc::fence_after_sync();
    return ok;
}

// Writes 32 consecutive bf16 columns [c0, c0+32) of row r into the A panels.
__device__ __forceinline__ void store_a_row32(uint32_t a_base, int r, int c0, const float (&v)[32]) {
    const int panel = c0 / kPanelElems;
    const int chunk0 = (c0 % kPanelElems) / 8;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
            w[e] = *reinterpret_cast<const uint32_t *>(&h2);
        }
        const uint32_t addr = a_base + panel * kPanelBytes + tc::sw128_offset(r, chunk0 + q);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                     "r"(w[3])
                     : "memory");
    }
}

struct TcMaps {
    CUtensorMap fwd[kMaxLayers];   // W_l      bf16 [W rows][din_p cols]
    CUtensorMap bwd[kMaxLayers];   // W_l^T    bf16 [din_p rows][W cols]
};

__global__ void __launch_bounds__(kTcThreads, 1)
    mlp_bf16_tc_kernel(const __grid_constant__ TcMaps maps, const float *__restrict__ X, int M, PotDev P,
                       float *__restrict__ E_mlp, float *__restrict__ dEdX, __nv_bfloat16 *__restrict__ scratch,
                       int *__restrict__ err) {
    extern __shared__ uint8_t smraw[];
    const uint32_t base = (tc::smem_u32(smraw) + 1023u) & ~1023u;
    TcSmem S;
    S.a = base;
    S.b0 = base + kMaxPanels * kPanelBytes;
    const uint32_t bars = S.b0 + 2 * kStageBytes;
    S.full0 = bars;
    S.empty0 = bars + 16;
    S.done = bars + 32;
    S.tslot = bars + 40;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int W = P.width, L = P.n_layers, d0p = P.d0p;
    const uint32_t ncols = 256;
    if (tid == 0) {
        tc::mbar_init(S.full(0), 1);
        tc::mbar_init(S.full(1), 1);
        tc::mbar_init(S.empty(0), 1);
        tc::mbar_init(S.empty(1), 1);
        tc::mbar_init(S.done, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(S.tslot, ncols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t tmem;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(S.tslot));
    const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t chunk = 0, gemm = 0;
    const int ntiles = (M + kTcRows - 1) / kTcRows;
    __nv_bfloat16 *my_scr = scratch + (size_t)blockIdx.x * L * kTcRows * W;
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row = tile * kTcRows + tid;
        const bool live = row < M;
        // input descriptors, fp32 -> bf16, into the A panels
        for (int c0 = 0; c0 < d0p; c0 += 32) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = live ? X[(size_t)row * d0p + c0 + i] : 0.f;
            store_a_row32(S.a, tid, c0, v);
        }
        tc::fence_async_shared();
        tc::fence_before_sync();
        __syncthreads();
        float y = 0.f;
        // forward
        int din = d0p;
        for (int l = 0; l < L && ok; ++l) {
            ok = tc_gemm(S, &maps.fwd[l], din, W, tmem, chunk, gemm);
            if (!__syncthreads_and(ok)) { ok = false; break; }
            const float *bl = P.b[l];
            __nv_bfloat16 *sp = my_scr + ((size_t)l * kTcRows + tid) * W;
            for (int c0 = 0; c0 < W; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tlane + c0, v);
#pragma unroll
                for (int i = 0; i < 32; i += 2) {
                    const float h0 = v[i] + bl[c0 + i], h1 = v[i + 1] + bl[c0 + i + 1];
                    v[i] = siluf_(h0);
                    v[i + 1] = siluf_(h1);
                    *reinterpret_cast<__nv_bfloat162 *>(sp + c0 + i) = __floats2bfloat162_rn(dsiluf_(h0), dsiluf_(h1));
                }
                if (l == L - 1) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) y += __bfloat162float(__float2bfloat16(v[i])) * P.wout[c0 + i];
                }
                store_a_row32(S.a, tid, c0, v);
            }
            tc::fence_async_shared();
            tc::fence_before_sync();
            __syncthreads();
            din = W;
        }
        if (!ok) break;
        // energy head
        y += P.bout;
        float dedy;
        if (P.head == LSD_HEAD_LINEAR) {
            if (live) E_mlp[row] = y;
            dedy = 1.f;
        } else {
            const float t = tanhf(y);
            if (live) E_mlp[row] = P.head_scale * t;
            dedy = P.head_scale * (1.f - t * t);
        }
        // g_L = e'(y) w_out * SiLU'(h_L)
        {
            const __nv_bfloat16 *sp = my_scr + ((size_t)(L - 1) * kTcRows + tid) * W;
            for (int c0 = 0; c0 < W; c0 += 32) {
                float v[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = dedy * P.wout[c0 + i] * __bfloat162float(sp[c0 + i]);
                store_a_row32(S.a, tid, c0, v);
            }
        }
        tc::fence_async_shared();
        tc::fence_before_sync();
        __syncthreads();
        // backward
        for (int l = L - 1; l >= 0 && ok; --l) {
            const int dout = l == 0 ? d0p : W;
            ok = tc_gemm(S, &maps.bwd[l], W, dout, tmem, chunk, gemm);
            if (!__syncthreads_and(ok)) { ok = false; break; }
            const __nv_bfloat16 *sp = my_scr + ((size_t)(l > 0 ? l - 1 : 0) * kTcRows + tid) * W;
            for (int c0 = 0; c0 < dout; c0 += 32) {
                float v[32];
                tc::tmem_ld32(tlane + c0, v);
                if (l > 0) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] *= __bfloat162float(sp[c0 + i]);
                    store_a_row32(S.a, tid, c0, v);
                } else if (live) {
                    float4 *dst = reinterpret_cast<float4 *>(dEdX + (size_t)row * d0p + c0);
#pragma unroll
                    for (int i = 0; i < 8; ++i) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                }
            }
            tc::fence_async_shared();
            tc::fence_before_sync();
            __syncthreads();
        }
        if (!ok) break;
    }
    if (!ok && tid == 0) atomicOr(err, 8);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct TcPlanImpl {
    TcMaps maps;
    bool ready = false;
};

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D bf16 tensor [rows][cols] (cols contiguous), box = 64 columns x box_rows rows, 128-byte swizzle.
static bool make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kPanelElems, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool mlp_tc_supported(const PotDev &P) {
    return P.has_mlp && P.width % 32 == 0 && P.width <= 256 && P.d0p <= 256 && P.n_layers <= kMaxLayers &&
           encode_fn() != nullptr;
}

size_t mlp_tc_smem_bytes() { return 1024 + kMaxPanels * kPanelBytes + 2 * kStageBytes + 64; }

size_t mlp_tc_scratch_elems(const PotDev &P, int n_cta) { return (size_t)n_cta * P.n_layers * kTcRows * P.width; }

void *mlp_tc_plan(const PotDev &P) {
    TcPlanImpl *pl = new TcPlanImpl();
    bool ok = true;
    for (int l = 0; l < P.n_layers && ok; ++l) {
        const int dinp = l == 0 ? P.d0p : P.width;
        ok = make_map(&pl->maps.fwd[l], P.Wn_bf[l], P.width, dinp, P.width) &&
             make_map(&pl->maps.bwd[l], P.Wt_bf[l], dinp, P.width, dinp);
    }
    pl->ready = ok;
    if (!ok) {
        delete pl;
        return nullptr;
    }
    return pl;
}

void mlp_tc_plan_free(void *plan) { delete (TcPlanImpl *)plan; }

int mlp_tc_grid(int M, int n_sm) {
    const int ntiles = (M + kTcRows - 1) / kTcRows;
    return ntiles < n_sm ? ntiles : n_sm;
}

void launch_mlp_tc(const void *plan, const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX,
                   __nv_bfloat16 *scratch, int n_sm, int *err, cudaStream_t s) {
    const TcPlanImpl *pl = (const TcPlanImpl *)plan;
    const int grid = mlp_tc_grid(M, n_sm);
    mlp_bf16_tc_kernel<<<grid, kTcThreads, mlp_tc_smem_bytes(), s>>>(pl->maps, X, M, P, E_mlp, dEdX, scratch, err);
}

cudaError_t mlp_tc_setup() {
    return cudaFuncSetAttribute(mlp_bf16_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mlp_tc_smem_bytes());
}

// ---------------------------------------------------------------------------
// FP32 potentials on the tensor cores: three TF32 products per term.
// Each FP32 operand x is split into x_hi = tf32(x) and x_lo = tf32(x - x_hi)
// (round to nearest), and every GEMM accumulates A_lo B_hi + A_hi B_lo +
// A_hi B_hi in the FP32 accumulator (the dropped A_lo B_lo term is below
// 2^-22 of the product), which keeps the result at FP32 accuracy.  Weights are
// split once on the host; activations in the epilogue.  32 FP32 elements per
// 128-byte swizzled row (K = 8 per instruction); A_hi and A_lo panels for K
// up to 128; three B stages, each holding the hi and lo chunks of 32
// K-columns, both copied by TMA against one mbarrier.
// Roles: warp 16 is the TMA producer and runs ahead through the whole GEMM
// sequence of the CTA's tiles (so the weights of the next GEMM land while the
// epilogue of the current one runs); thread 0 issues the MMAs; the 16 warps
// 0..15 run the epilogues, warp w reading TMEM lane quarter w % 4 (rows
// 32 (w % 4) + lane) and column block w / 4 (32 columns).  TMEM columns
// [0, 128) hold the accumulator and columns 128 + l W + c hold SiLU'(h_l) of
// the tile's rows (written by tcgen05.st in the forward epilogues, read back
// in the backward ones), so nothing of a tile leaves the SM but dE/dX and E.
// ---------------------------------------------------------------------------
constexpr int kTfPanelElems = 32;                  // FP32 elements per 128-byte swizzled row
constexpr int kTfMaxPanels = 4;                    // K up to 128
constexpr int kTfChunkBytes = 128 * 128;           // one B chunk (hi or lo): up to 128 rows x 128 B
constexpr int kTfStages = 3;
constexpr uint32_t kTfTmemCols = 512;              // accumulator (N up to 128) + SiLU' of L layers
constexpr int kTfAccCols = 128;
constexpr int kTfEpiWarps = 16;
constexpr int kTfEpiThreads = kTfEpiWarps * 32;
constexpr int kTfThreads = kTfEpiThreads + 32;     // + the TMA producer warp

// Shared-memory addresses; per-stage ones are computed, not stored in arrays
// (a runtime-indexed array would live in local memory).
struct TfSmem {
    uint32_t ahi, alo;     // A operand panels
    uint32_t b0;           // stage s: hi chunk at b0 + 2 s C, lo chunk C after it
    uint32_t full0, empty0, done, tslot;
    float *ypart;          // [3][128] partial head sums of column blocks 1..3
    __device__ __forceinline__ uint32_t bhi(int s) const { return b0 + (uint32_t)s * 2u * kTfChunkBytes; }
    __device__ __forceinline__ uint32_t blo(int s) const { return bhi(s) + kTfChunkBytes; }
    __device__ __forceinline__ uint32_t full(int s) const { return full0 + 8u * (uint32_t)s; }
    __device__ __forceinline__ uint32_t empty(int s) const { return empty0 + 8u * (uint32_t)s; }
};

// barrier 1: the epilogue warps only (the producer warp runs on its own)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTfEpiThreads) : "memory"); }
__device__ __forceinline__ bool epi_and(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kTfEpiThreads)
        : "memory");
    return r != 0;
}

// The MMAs of one GEMM (thread 0), then every epilogue thread waits for the
// accumulator.  chunk counts B chunks over the kernel (stage = chunk % 3,
// use = chunk / 3), in the producer's order; gemm counts GEMMs.
__device__ __forceinline__ bool tf_mma(const TfSmem &S, int K, int N, uint32_t tmem, uint32_t &chunk, uint32_t &gemm) {
    bool ok = true;
    const int nk = (K + kTfPanelElems - 1) / kTfPanelElems;
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        const uint32_t idesc = tc::idesc_f32acc(tc::kFmtTF32, kTcRows, N);
        for (int kc = 0; kc < nk; ++kc) {
            const uint32_t c = chunk + kc;
            const int s = c % kTfStages;
            if (!tc::mbar_wait(S.full(s), (c / kTfStages) & 1)) { ok = false; break; }
            tc::fence_after_sync();
            const int kend = min(kTfPanelElems, K - kc * kTfPanelElems);
            for (int k8 = 0; k8 < kend; k8 += 8) {
                const uint32_t ao = kc * kPanelBytes + k8 * 4;
                const uint64_t ahd = tc::sdesc_sw128(S.ahi + ao), ald = tc::sdesc_sw128(S.alo + ao);
                const uint64_t bhd = tc::sdesc_sw128(S.bhi(s) + k8 * 4), bld = tc::sdesc_sw128(S.blo(s) + k8 * 4);
                tc::mma_tf32(tmem, ald, bhd, idesc, (kc | k8) != 0);
                tc::mma_tf32(tmem, ahd, bld, idesc, 1u);
                tc::mma_tf32(tmem, ahd, bhd, idesc, 1u);
            }
            tc::mma_commit(S.empty(s));
        }
        if (ok) tc::mma_commit(S.done);
    }
    chunk += nk;
    if (!tc::mbar_wait(S.done, gemm & 1)) ok = false;
    ++gemm;
    tc::fence_after_sync();
    return ok;
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Writes the hi and lo TF32 parts of NC (16 or 32) consecutive FP32 columns
// [c0, c0 + NC) of row r; c0 is a multiple of 16 (half or all of the
// swizzled row of panel c0 / 32).
template <int NC>
__device__ __forceinline__ void store_split_row(uint32_t ahi, uint32_t alo, int r, int c0, const float (&v)[NC]) {
    const int panel = c0 / kTfPanelElems, q0 = (c0 % kTfPanelElems) / 4;
#pragma unroll
    for (int qq = 0; qq < NC / 4; ++qq) {
        const int q = q0 + qq;
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float x = v[4 * qq + e];
            h[e] = tf32_rna(x);
            l[e] = tf32_rna(x - __uint_as_float(h[e]));
        }
        const uint32_t off = panel * kPanelBytes + tc::sw128_offset(r, q);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ahi + off), "r"(h[0]), "r"(h[1]), "r"(h[2]),
                     "r"(h[3])
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(alo + off), "r"(l[0]), "r"(l[1]), "r"(l[2]),
                     "r"(l[3])
                     : "memory");
    }
}

struct TfMaps {
    CUtensorMap fwd_hi[kMaxLayers], fwd_lo[kMaxLayers];   // W_l   [W rows][din_p cols]
    CUtensorMap bwd_hi[kMaxLayers], bwd_lo[kMaxLayers];   // W_l^T [din_p rows][W cols]
};

// The TMA producer: B chunks of every GEMM of the CTA's tiles, in the order
// the MMAs consume them, at most kTfStages ahead.  Before returning it waits
// for the landing of the copies it issued, so none is in flight at exit.
__device__ void tf_producer(const TfSmem &S, const TfMaps &maps, int M, const PotDev &P, int *err) {
    const int W = P.width, L = P.n_layers, d0p = P.d0p;
    const int ntiles = (M + kTcRows - 1) / kTcRows;
    uint32_t c = 0;
    bool ok = true;
    auto gemm_chunks = [&](const CUtensorMap *mhi, const CUtensorMap *mlo, int K, int N) {
        const int nk = (K + kTfPanelElems - 1) / kTfPanelElems;
        for (int kc = 0; kc < nk && ok; ++kc, ++c) {
            const int s = c % kTfStages;
            if (c >= (uint32_t)kTfStages && !tc::mbar_wait(S.empty(s), ((c / kTfStages) - 1) & 1)) {
                ok = false;
                break;
            }
            tc::mbar_expect_tx(S.full(s), 2u * (uint32_t)N * 128u);
            tc::tma_load_2d(S.bhi(s), mhi, kc * kTfPanelElems, 0, S.full(s));
            tc::tma_load_2d(S.blo(s), mlo, kc * kTfPanelElems, 0, S.full(s));
        }
    };
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int l = 0; l < L && ok; ++l) gemm_chunks(&maps.fwd_hi[l], &maps.fwd_lo[l], l == 0 ? d0p : W, W);
        for (int l = L - 1; l >= 0 && ok; --l) gemm_chunks(&maps.bwd_hi[l], &maps.bwd_lo[l], W, l == 0 ? d0p : W);
    }
    // the copies of the last (up to kTfStages) chunks issued
    const uint32_t first = c > (uint32_t)kTfStages ? c - kTfStages : 0u;
    for (uint32_t k = first; k < c; ++k)
        if (!tc::mbar_wait(S.full(k % kTfStages), (k / kTfStages) & 1)) ok = false;
    if (!ok) atomicOr(err, 8);
}

__global__ void __launch_bounds__(kTfThreads, 1)
    mlp_tf32x3_tc_kernel(const __grid_constant__ TfMaps maps, const float *__restrict__ X, int M, PotDev P,
                         float *__restrict__ E_mlp, float *__restrict__ dEdX, int *__restrict__ err) {
    extern __shared__ uint8_t smraw[];
    const uint32_t base = (tc::smem_u32(smraw) + 1023u) & ~1023u;
    TfSmem S;
    S.ahi = base;
    S.alo = S.ahi + kTfMaxPanels * kPanelBytes;
    S.b0 = S.alo + kTfMaxPanels * kPanelBytes;
    const uint32_t at = S.b0 + 2 * kTfStages * kTfChunkBytes;
    S.full0 = at;
    S.empty0 = at + 8 * kTfStages;
    S.done = at + 16 * kTfStages;
    S.tslot = S.done + 8;
    S.ypart = reinterpret_cast<float *>(smraw + (S.tslot + 8 - tc::smem_u32(smraw)));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int W = P.width, L = P.n_layers, d0p = P.d0p;
    if (tid == 0) {
        for (int st = 0; st < kTfStages; ++st) {
            tc::mbar_init(S.full(st), 1);
            tc::mbar_init(S.empty(st), 1);
        }
        tc::mbar_init(S.done, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(S.tslot, kTfTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    uint32_t tmem;
    asm volatile("ld.shared.b32 %0, [%1];" : "=r"(tmem) : "r"(S.tslot));
    if (warp == kTfEpiWarps) {
        if (lane == 0) tf_producer(S, maps, M, P, err);
    } else {
        const int quarter = warp & 3, cb = warp >> 2, c0 = 32 * cb;
        const int r = 32 * quarter + lane;                      // row in the tile
        const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0;
        uint32_t chunk = 0, gemm = 0;
        const int ntiles = (M + kTcRows - 1) / kTcRows;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int row = tile * kTcRows + r;
            const bool live = row < M;
            if (c0 < d0p) {
                float v[32];
                if (live) {
                    const float4 *src = reinterpret_cast<const float4 *>(X + (size_t)row * d0p + c0);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 t = src[i];
                        v[4 * i] = t.x;
                        v[4 * i + 1] = t.y;
                        v[4 * i + 2] = t.z;
                        v[4 * i + 3] = t.w;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = 0.f;
                }
                store_split_row<32>(S.ahi, S.alo, r, c0, v);
            }
            tc::fence_async_shared();
            tc::fence_before_sync();
            epi_sync();
            float y = 0.f;
            int din = d0p;
            for (int l = 0; l < L; ++l) {
                ok = epi_and(tf_mma(S, din, W, tmem, chunk, gemm));
                if (!ok) break;
                if (c0 < W) {
                    const float4 *bl = reinterpret_cast<const float4 *>(layer_bias(P, l) + c0);
#pragma unroll 1
                    for (int hf = 0; hf < 2; ++hf) {
                        float v[16], d[16];
                        tc::tmem_ld16(taddr + 16 * hf, v);
#pragma unroll
                        for (int i = 0; i < 16; i += 4) {
                            const float4 b4 = __ldg(bl + 4 * hf + i / 4);
                            silu_dsilu_fast(v[i] + b4.x, v[i], d[i]);
                            silu_dsilu_fast(v[i + 1] + b4.y, v[i + 1], d[i + 1]);
                            silu_dsilu_fast(v[i + 2] + b4.z, v[i + 2], d[i + 2]);
                            silu_dsilu_fast(v[i + 3] + b4.w, v[i + 3], d[i + 3]);
                        }
                        tc::tmem_st16(taddr + kTfAccCols + l * W + 16 * hf, d);
                        if (l == L - 1) {
#pragma unroll
                            for (int i = 0; i < 16; ++i) y += v[i] * P.wout[c0 + 16 * hf + i];
                        }
                        store_split_row<16>(S.ahi, S.alo, r, c0 + 16 * hf, v);
                    }
                    if (l == L - 1 && cb > 0) S.ypart[(cb - 1) * kTcRows + r] = y;
                }
                tc::fence_async_shared();
                tc::fence_before_sync();
                epi_sync();
                din = W;
            }
            if (!ok) break;
            // energy head (column block 0 holds the row's sum), e'(y) to every column block
            if (cb == 0) {
                for (int b = 1; b < W / 32; ++b) y += S.ypart[(b - 1) * kTcRows + r];
                y += P.bout;
                float dedy;
                if (P.head == LSD_HEAD_LINEAR) {
                    if (live) E_mlp[row] = y;
                    dedy = 1.f;
                } else {
                    const float t = tanhf(y);
                    if (live) E_mlp[row] = P.head_scale * t;
                    dedy = P.head_scale * (1.f - t * t);
                }
                S.ypart[r] = dedy;
            }
            epi_sync();
            const float dedy = S.ypart[r];
            if (c0 < W) {
                float v[32];
                tc::tmem_ld32(taddr + kTfAccCols + (L - 1) * W, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] *= dedy * P.wout[c0 + i];
                store_split_row<32>(S.ahi, S.alo, r, c0, v);
            }
            tc::fence_async_shared();
            tc::fence_before_sync();
            epi_sync();
            for (int l = L - 1; l >= 0; --l) {
                const int dout = l == 0 ? d0p : W;
                ok = epi_and(tf_mma(S, W, dout, tmem, chunk, gemm));
                if (!ok) break;
                if (c0 < dout) {
                    float v[32];
                    tc::tmem_ld32(taddr, v);
                    if (l > 0) {
                        float d[32];
                        tc::tmem_ld32(taddr + kTfAccCols + (l - 1) * W, d);
#pragma unroll
                        for (int i = 0; i < 32; ++i) v[i] *= d[i];
                        store_split_row<32>(S.ahi, S.alo, r, c0, v);
                    } else if (live) {
                        float4 *dst = reinterpret_cast<float4 *>(dEdX + (size_t)row * d0p + c0);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                    }
                }
                tc::fence_async_shared();
                tc::fence_before_sync();
                epi_sync();
            }
        }
        if (!ok && tid == 0) atomicOr(err, 8);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTfTmemCols);
}

struct TfPlanImpl {
    TfMaps maps;
};

// 2-D FP32 tensor [rows][cols] (cols contiguous), box = 32 columns x box_rows rows, 128-byte swizzle.
static bool make_map_f32(CUtensorMap *m, const void *ptr, int rows, int cols, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
    cuuint32_t box[2] = {(cuuint32_t)kTfPanelElems, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool mlp_tf32_supported(const PotDev &P) {
    return P.has_mlp && P.width % 32 == 0 && P.width <= 128 && P.d0p <= 128 && P.n_layers <= kMaxLayers &&
           kTfAccCols + P.n_layers * P.width <= (int)kTfTmemCols && encode_fn() != nullptr;
}

size_t mlp_tf32_smem_bytes() {
    return 1024 + 2 * kTfMaxPanels * kPanelBytes + 2 * kTfStages * kTfChunkBytes + 128 + 3 * kTcRows * sizeof(float);
}

void *mlp_tf32_plan(const PotDev &P, const Tf32Weights &w) {
    TfPlanImpl *pl = new TfPlanImpl();
    bool ok = true;
    for (int l = 0; l < P.n_layers && ok; ++l) {
        const int dinp = l == 0 ? P.d0p : P.width;
        ok = make_map_f32(&pl->maps.fwd_hi[l], w.wn_hi[l], P.width, dinp, P.width) &&
             make_map_f32(&pl->maps.fwd_lo[l], w.wn_lo[l], P.width, dinp, P.width) &&
             make_map_f32(&pl->maps.bwd_hi[l], w.wt_hi[l], dinp, P.width, dinp) &&
             make_map_f32(&pl->maps.bwd_lo[l], w.wt_lo[l], dinp, P.width, dinp);
    }
    if (!ok) {
        delete pl;
        return nullptr;
    }
    return pl;
}

void mlp_tf32_plan_free(void *plan) { delete (TfPlanImpl *)plan; }

void launch_mlp_tf32(const void *plan, const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX, int n_sm,
                     int *err, cudaStream_t s) {
    const TfPlanImpl *pl = (const TfPlanImpl *)plan;
    const int grid = mlp_tc_grid(M, n_sm);
    mlp_tf32x3_tc_kernel<<<grid, kTfThreads, mlp_tf32_smem_bytes(), s>>>(pl->maps, X, M, P, E_mlp, dEdX, err);
}

cudaError_t mlp_tf32_setup() {
    return cudaFuncSetAttribute(mlp_tf32x3_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mlp_tf32_smem_bytes());
}

// ---------------------------------------------------------------------------
// The same kernel for callers that cannot allocate device memory: its SiLU'
// scratch is this file-scope array (4 MiB, held by every device that loads the
// library until the process exits) instead of a slot the handle allocated.
// Nothing in it has to start at zero: each CTA writes a row's SiLU' values
// before reading them.  All calls share the array, so calls that overlap on
// the GPU (two streams, two handles) race on it.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = (size_t)4 << 20;
constexpr size_t kStaticScratchElems = kStaticScratchBytes / sizeof(__nv_bfloat16);
static __device__ __align__(256) __nv_bfloat16 g_static_mlp_scratch[kStaticScratchElems];

constexpr int kStaticMaxDevices = 64;
static void *g_static_scratch_addr[kStaticMaxDevices];   // device address of the array, per device

size_t mlp_tc_static_scratch_bytes() { return kStaticScratchBytes; }

int mlp_tc_static_launch(const void *plan, const float *X, int M, const PotDev &P, float *E_mlp, float *dEdX,
                         int n_sm, int *err, cudaStream_t s) {
    const size_t per_cta = (size_t)P.n_layers * kTcRows * P.width;
    if (per_cta > kStaticScratchElems) return LSD_EINVAL;   // one tile's SiLU' does not fit the array
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return LSD_ECUDA;
    if (!g_static_scratch_addr[dev]) {
        // set-up, once per device, with that device current: the host-side name
        // of the array is not a device address; ask the runtime for it
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_mlp_scratch) != cudaSuccess || !p) return LSD_ECUDA;
        g_static_scratch_addr[dev] = p;
    }
    const int cap = (int)(kStaticScratchElems / per_cta);
    int grid = mlp_tc_grid(M, n_sm);
    if (grid > cap) grid = cap;
    const TcPlanImpl *pl = (const TcPlanImpl *)plan;
    mlp_bf16_tc_kernel<<<grid, kTcThreads, mlp_tc_smem_bytes(), s>>>(
        pl->maps, X, M, P, E_mlp, dEdX, (__nv_bfloat16 *)g_static_scratch_addr[dev], err);
    return cudaGetLastError() == cudaSuccess ? LSD_OK : LSD_ECUDA;
}

}  // namespace lsd

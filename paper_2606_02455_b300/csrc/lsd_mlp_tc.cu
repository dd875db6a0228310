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
    uint32_t b[2];       // B stages
    uint32_t full[2];    // TMA landed
    uint32_t empty[2];   // MMAs done with the stage
    uint32_t done;       // all MMAs of a GEMM done
    uint32_t tslot;      // TMEM base address
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
            if (c >= 2 && ok) ok = tc::mbar_wait(S.empty[s], ((c >> 1) - 1) & 1);
            if (!ok) return;
            tc::mbar_expect_tx(S.full[s], bytes);
            tc::tma_load_2d(S.b[s], map, kc * kPanelElems, 0, S.full[s]);
        };
        const uint32_t c0 = chunk;
        issue(c0, 0);
        for (int kc = 0; kc < nk && ok; ++kc) {
            const uint32_t c = c0 + kc;
            if (kc + 1 < nk) issue(c + 1, kc + 1);
            const int s = c & 1;
            if (!tc::mbar_wait(S.full[s], (c >> 1) & 1)) { ok = false; break; }
            tc::fence_after_sync();
            const int kend = min(kPanelElems, K - kc * kPanelElems);
            for (int k16 = 0; k16 < kend; k16 += 16) {
                const uint64_t ad = tc::sdesc_sw128(S.a + kc * kPanelBytes + k16 * 2);
                const uint64_t bd = tc::sdesc_sw128(S.b[s] + k16 * 2);
                tc::mma_f16(tmem, ad, bd, idesc, (kc | k16) != 0);
            }
            tc::mma_commit(S.empty[s]);
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
    S.b[0] = base + kMaxPanels * kPanelBytes;
    S.b[1] = S.b[0] + kStageBytes;
    const uint32_t bars = S.b[1] + kStageBytes;
    S.full[0] = bars;
    S.full[1] = bars + 8;
    S.empty[0] = bars + 16;
    S.empty[1] = bars + 24;
    S.done = bars + 32;
    S.tslot = bars + 40;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int W = P.width, L = P.n_layers, d0p = P.d0p;
    const uint32_t ncols = 256;
    if (tid == 0) {
        tc::mbar_init(S.full[0], 1);
        tc::mbar_init(S.full[1], 1);
        tc::mbar_init(S.empty[0], 1);
        tc::mbar_init(S.empty[1], 1);
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

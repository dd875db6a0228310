// lsd_verlet.cu -- per-window Verlet candidate lists from a cell grid.
//
// At the start of every window (and of every plain step) the base positions
// are binned into a cell grid with cells at least r_list = r_cut + skin wide,
// and every atom gets the sorted list of atoms whose minimum image lies within
// r_list.  The draft then verifies, at every step, that no atom has moved more
// than 0.45 skin from the base (otherwise it stops drafting: the window is
// truncated at that step), so for every drafted step each pair within r_cut
// is in the list; every list entry is still tested with the exact membership
// rule, so the interacting sets are exactly the rule's.
//
// cell_count_kernel   fixed point of the base positions, cell of each atom, counts
// cell_scan_kernel    exclusive scan of the counts (one CTA)
// cell_fill_kernel    atom indices in cell order (slot order inside a cell does
//                     not matter: lists are sorted afterwards)
// verlet_list_kernel  one warp per atom: 27 neighbouring cells (or all atoms
//                     for a grid narrower than 3 cells), minimum-image test,
//                     compaction in shared memory, a bitonic sort in registers
//                     (up to 512 candidates) and the sorted list out
// verlet_check_kernel lists kept across windows: whether this window needs new
//                     lists (the build kernels return at once otherwise)
#include "lsd_common.cuh"
#include "lsd_kernels.h"

namespace lsd {

__device__ __forceinline__ int cell_of(uint32_t u, int nc) { return (int)(((unsigned long long)u * (unsigned)nc) >> 32); }

__global__ void cell_count_kernel(const double *__restrict__ q, const int *__restrict__ species, Geo g, int3 nc,
                                  uint4 *__restrict__ fix_base, int *__restrict__ cell_of_atom,
                                  int *__restrict__ cell_count, const int *__restrict__ skip,
                                  const int *__restrict__ rebuild) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.N || (skip && *skip) || (rebuild && !*rebuild)) return;
    const uint32_t ux = fixpoint(q[3 * i], g.scale[0]), uy = fixpoint(q[3 * i + 1], g.scale[1]),
                   uz = fixpoint(q[3 * i + 2], g.scale[2]);
    fix_base[i] = make_uint4(ux, uy, uz, (unsigned)species[i]);
    const int c = (cell_of(uz, nc.z) * nc.y + cell_of(uy, nc.y)) * nc.x + cell_of(ux, nc.x);
    cell_of_atom[i] = c;
    atomicAdd(&cell_count[c], 1);
}

__global__ void cell_scan_kernel(int ncells, int *__restrict__ cell_count, int *__restrict__ cell_start,
                                 const int *__restrict__ skip, const int *__restrict__ rebuild) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if ((skip && *skip) || (rebuild && !*rebuild)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ncells; base += blockDim.x) {
        const int c = base + threadIdx.x;
        const int v = c < ncells ? cell_count[c] : 0;
        int s = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane == 31) warp_tot[w] = s;
        __syncthreads();
        if (w == 0) {
            int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += u;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        const int excl = carry + (w > 0 ? warp_tot[w - 1] : 0) + s - v;
        if (c < ncells) {
            cell_start[c] = excl;
            cell_count[c] = 0;   // reused as the fill cursor
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) cell_start[ncells] = carry;
}

__global__ void cell_fill_kernel(int N, const int *__restrict__ cell_of_atom, const int *__restrict__ cell_start,
                                 int *__restrict__ cursor, int *__restrict__ cell_atoms, const int *__restrict__ skip,
                                 const int *__restrict__ rebuild) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N || (skip && *skip) || (rebuild && !*rebuild)) return;
    const int c = cell_of_atom[i];
    cell_atoms[cell_start[c] + atomicAdd(&cursor[c], 1)] = i;
}

// Sorts 32 E keys held E per lane (key e = r * 32 + lane in v[r]) in
// ascending order with a bitonic network: partners 32 or more apart are in the
// same lane (register compare-exchange), nearer ones one shuffle away.
template <int E>
__device__ __forceinline__ void warp_bitonic_sort(int (&v)[E], int lane) {
#pragma unroll
    for (int k = 2; k <= 32 * E; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jj = j >> 5;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    if (r & jj) continue;
                    const bool up = ((r * 32) & k) == 0;
                    const int a = v[r], b = v[r | jj];
                    v[r] = up ? min(a, b) : max(a, b);
                    v[r | jj] = up ? max(a, b) : min(a, b);
                }
            } else {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const bool up = ((r * 32 + lane) & k) == 0;
                    const int o = __shfl_xor_sync(0xffffffffu, v[r], j);
                    v[r] = (((lane & j) == 0) == up) ? min(v[r], o) : max(v[r], o);
                }
            }
        }
    }
}

// The n compacted candidates of buf, sorted, to out (coalesced).
template <int E>
__device__ __forceinline__ void sort_out(const int *buf, int n, int *out, int lane) {
    int v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) v[r] = r * 32 + lane < n ? buf[r * 32 + lane] : 0x7fffffff;
    warp_bitonic_sort<E>(v, lane);
#pragma unroll
    for (int r = 0; r < E; ++r)
        if (r * 32 + lane < n) out[r * 32 + lane] = v[r];
}

__global__ void verlet_list_kernel(const uint4 *__restrict__ fix_base, const int *__restrict__ cell_of_atom,
                                   const int *__restrict__ cell_start, const int *__restrict__ cell_atoms, Geo g,
                                   int3 nc, float rlist2f, int cap, int cap_pow2, int *__restrict__ vlist,
                                   int *__restrict__ vcount, DevState *st, const int *__restrict__ skip,
                                   const int *__restrict__ rebuild) {
    extern __shared__ int sbuf[];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= g.N || (skip && *skip) || (rebuild && !*rebuild)) return;
    int *buf = sbuf + (size_t)wib * cap_pow2;
    const uint4 fi = fix_base[i];
    const bool one_cell = nc.x < 3 || nc.y < 3 || nc.z < 3;
    const int ci = cell_of_atom[i];
    const int cx = ci % nc.x, cy = (ci / nc.x) % nc.y, cz = ci / (nc.x * nc.y);
    int cnt = 0;
    const int ncell_scan = one_cell ? 1 : 27;
    const unsigned below = (1u << lane) - 1u;
    for (int t = 0; t < ncell_scan; ++t) {
        int s0, s1;
        if (one_cell) {
            s0 = 0;
            s1 = g.N;
        } else {
            const int ox = t % 3 - 1, oy = (t / 3) % 3 - 1, oz = t / 9 - 1;
            const int c = (((cz + oz + nc.z) % nc.z) * nc.y + (cy + oy + nc.y) % nc.y) * nc.x + (cx + ox + nc.x) % nc.x;
            s0 = cell_start[c];
            s1 = cell_start[c + 1];
        }
        // four candidates per lane in flight: their loads first, then the tests
        constexpr int kB = 4;
        for (int base = s0; base < s1; base += 32 * kB) {
            int kk[kB];
            uint4 fk[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int p = base + 32 * u + lane;
                kk[u] = p < s1 ? (one_cell ? p : cell_atoms[p]) : -1;
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) fk[u] = kk[u] >= 0 ? fix_base[kk[u]] : fi;
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                if (base + 32 * u >= s1) break;
                bool in = false;
                if (kk[u] >= 0 && kk[u] != i) {
                    float dx, dy, dz;
                    int kx;
                    axis_min(fi.x, fk[u].x, g.scale_f[0], dx, kx);
                    axis_min(fi.y, fk[u].y, g.scale_f[1], dy, kx);
                    axis_min(fi.z, fk[u].z, g.scale_f[2], dz, kx);
                    in = dist2_rule(dx, dy, dz) < rlist2f;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                const int pos = cnt + __popc(bal & below);
                if (in && pos < cap_pow2) buf[pos] = kk[u];
                cnt += __popc(bal);
            }
        }
    }
    // (an atom's own images lie at least one box length away, beyond any cutoff rc < L)
    const int n = cnt < cap ? cnt : cap;
    __syncwarp();
    int *out = vlist + (size_t)i * cap;
    if (one_cell) {
        // a single-cell scan runs in index order: already sorted
        for (int p = lane; p < n; p += 32) out[p] = buf[p];
    } else if (n <= 32) {
        sort_out<1>(buf, n, out, lane);
    } else if (n <= 64) {
        sort_out<2>(buf, n, out, lane);
    } else if (n <= 128) {
        sort_out<4>(buf, n, out, lane);
    } else if (n <= 256) {
        sort_out<8>(buf, n, out, lane);
    } else if (n <= 512) {
        sort_out<16>(buf, n, out, lane);
    } else {
        // longer lists: a bitonic sort of cap_pow2 entries in shared memory
        for (int p = n + lane; p < cap_pow2; p += 32) buf[p] = 0x7fffffff;
        __syncwarp();
        for (int k2 = 2; k2 <= cap_pow2; k2 <<= 1) {
            for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                for (int a = lane; a < cap_pow2; a += 32) {
                    const int b = a ^ j2;
                    if (b > a) {
                        const int x = buf[a], y = buf[b];
                        const bool up = (a & k2) == 0;
                        if (up ? x > y : x < y) {
                            buf[a] = y;
                            buf[b] = x;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int p = lane; p < n; p += 32) out[p] = buf[p];
    }
    if (lane == 0) {
        vcount[i] = n;
        if (cnt > cap) atomicOr(&st->err, 1);
    }
}

// skip (device, may be null): when it points at a nonzero flag every kernel
// returns at once (the pipelined loop keeps an already valid draft).
// Lists kept across windows (and plain steps): the blocks compare positions
// with the lists' base (the fixed point of the draft's displacement check) and
// the last block to finish decides whether the lists are rebuilt: when some
// atom has moved more than sqrt(keep2f), or the last window ended at the
// draft's displacement bound (list_force).  The lists stay correct either way:
// the draft checks every drafted step against the same base and stops at the
// bound.
__global__ void verlet_check_kernel(const double *__restrict__ q, const uint4 *__restrict__ fix_base, Geo g,
                                    float keep2f, DevState *st) {
    __shared__ bool s_last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool moved = false;
    if (i < g.N) {
        const uint4 b = fix_base[i];
        float d, d2;
        int kk;
        axis_min(b.x, fixpoint(q[3 * i], g.scale[0]), g.scale_f[0], d, kk);
        d2 = d * d;
        axis_min(b.y, fixpoint(q[3 * i + 1], g.scale[1]), g.scale_f[1], d, kk);
        d2 += d * d;
        axis_min(b.z, fixpoint(q[3 * i + 2], g.scale[2]), g.scale_f[2], d, kk);
        d2 += d * d;
        moved = d2 > keep2f;
    }
    const int any = __syncthreads_or(moved);
    if (threadIdx.x == 0) {
        if (any) atomicOr(&st->list_moved, 1);
        __threadfence();
        s_last = atomicAdd(&st->list_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const int rebuild = (atomicOr(&st->list_moved, 0) || st->list_force) ? 1 : 0;
        st->list_rebuild = rebuild;
        st->list_moved = 0;
        st->list_force = 0;
        st->list_done = 0u;
        st->list_builds += rebuild;
    }
}

void launch_verlet_check(const double *q, const VerletBufs &b, const Geo &g, float keep2f, DevState *st,
                         cudaStream_t s) {
    verlet_check_kernel<<<(g.N + 255) / 256, 256, 0, s>>>(q, b.fix_base, g, keep2f, st);
}

void launch_verlet_build(const VerletPlan &vp, const double *q, const int *species, const Geo &g, VerletBufs &b,
                         DevState *st, cudaStream_t s, const int *skip, const int *rebuild) {
    const int N = g.N;
    const int3 nc = make_int3(vp.nc[0], vp.nc[1], vp.nc[2]);
    const int ncells = vp.nc[0] * vp.nc[1] * vp.nc[2];
    const bool one_cell = vp.nc[0] < 3 || vp.nc[1] < 3 || vp.nc[2] < 3;
    if (!one_cell) cudaMemsetAsync(b.cell_count, 0, (size_t)ncells * sizeof(int), s);
    cell_count_kernel<<<(N + 255) / 256, 256, 0, s>>>(q, species, g, one_cell ? make_int3(1, 1, 1) : nc, b.fix_base,
                                                       b.cell_of_atom, one_cell ? b.cell_scratch : b.cell_count, skip,
                                                       rebuild);
    if (!one_cell) {
        cell_scan_kernel<<<1, 1024, 0, s>>>(ncells, b.cell_count, b.cell_start, skip, rebuild);
        cell_fill_kernel<<<(N + 255) / 256, 256, 0, s>>>(N, b.cell_of_atom, b.cell_start, b.cell_count, b.cell_atoms,
                                                          skip, rebuild);
    }
    const int warps = 8;
    verlet_list_kernel<<<(N + warps - 1) / warps, warps * 32, (size_t)warps * vp.cap_pow2 * sizeof(int), s>>>(
        b.fix_base, b.cell_of_atom, b.cell_start, b.cell_atoms, g, nc, vp.rlist2f, vp.cap, vp.cap_pow2, b.vlist,
        b.vcount, st, skip, rebuild);
}

cudaError_t verlet_setup(int max_smem) {
    return cudaFuncSetAttribute(verlet_list_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

}  // namespace lsd

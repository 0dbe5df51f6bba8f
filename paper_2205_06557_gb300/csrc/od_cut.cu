// Ion-ion forces with a cutoff (Sec. 5: a switching function that vanishes beyond a
// fixed distance, so that distant ion pairs cost nothing).
//
// Every evaluation:
//   1. the ions are sorted stably by z-slab (slab width a fraction of the cutoff): a
//      counting sort whose blocks are single warps, so the rank of an ion among the
//      ions of its slab in the same warp comes from __match_any_sync, and the order
//      inside a slab is the ion order (deterministic);
//   2. the sorted positions are cut into tiles of TI ions; each tile gets the bounding
//      box of its ions;
//   3. warps list, for every tile I, the tiles J >= I whose boxes come closer than the
//      cutoff (the tile pairs to evaluate);
//   4. persistent CTAs evaluate those tile pairs with the symmetric packed-pair unit of
//      the all-pairs kernel and the switched pair coefficient (the plain one where the
//      two boxes lie wholly inside the switching distance); a pair beyond the cutoff
//      inside a listed tile pair contributes exactly zero; the sums go to the fixed-point
//      accumulators at the ions' sorted positions;
//   5. the kick reads, for ion i, the accumulator of its sorted position.
// Nothing is read back to the host, so the step stays one CUDA graph.
#include <algorithm>
#include <cmath>

#include "od_device.cuh"

namespace od {

constexpr int CUT_SCAN_PER = 8;                 // elements per thread in the block scan
constexpr int CUT_SCAN_CHUNK = 1024 * CUT_SCAN_PER;

__device__ __forceinline__ int slab_of(float z, float zoff, float inv_w, int nslab)
{
    return min(max((int)((z + zoff) * inv_w), 0), nslab - 1);
}

// per-warp slab counts: bcount[slab * nblk + warp] (zeroed before)
__global__ void k_cut_hist(const float4* __restrict__ fpos, int N, float zoff, float inv_w, int nslab, int nblk,
                           int* __restrict__ bcount)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int key = i < N ? slab_of(fpos[i].z, zoff, inv_w, nslab) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && lane == __ffs(peers) - 1) bcount[(long long)key * nblk + (i >> 5)] = __popc(peers);
}

// exclusive scan of n ints, chunks of CUT_SCAN_CHUNK per 1024-thread block
__device__ __forceinline__ int block_excl_scan(int v, int* s_w, int& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s_w[lane] = t;
    }
    __syncthreads();
    total = s_w[(blockDim.x >> 5) - 1];
    const int before = w > 0 ? s_w[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void k_cut_scan_chunks(const int* __restrict__ in, int* __restrict__ out, long long n, int* __restrict__ bsum)
{
    __shared__ int s_w[32];
    const long long base = (long long)blockIdx.x * CUT_SCAN_CHUNK + (long long)threadIdx.x * CUT_SCAN_PER;
    int v[CUT_SCAN_PER], sum = 0;
#pragma unroll
    for (int k = 0; k < CUT_SCAN_PER; ++k) {
        v[k] = base + k < n ? in[base + k] : 0;
        sum += v[k];
    }
    int total;
    int run = block_excl_scan(sum, s_w, total);
#pragma unroll
    for (int k = 0; k < CUT_SCAN_PER; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

// exclusive scan of the chunk sums in one block (nb <= 1024 * CUT_SCAN_PER), then added
__global__ void k_cut_scan_sums(int* __restrict__ bsum, int nb)
{
    __shared__ int s_w[32];
    int v[CUT_SCAN_PER], sum = 0;
    const int base = threadIdx.x * CUT_SCAN_PER;
#pragma unroll
    for (int k = 0; k < CUT_SCAN_PER; ++k) {
        v[k] = base + k < nb ? bsum[base + k] : 0;
        sum += v[k];
    }
    int total;
    int run = block_excl_scan(sum, s_w, total);
#pragma unroll
    for (int k = 0; k < CUT_SCAN_PER; ++k) {
        if (base + k < nb) bsum[base + k] = run;
        run += v[k];
    }
}

__global__ void k_cut_scan_add(int* __restrict__ out, long long n, const int* __restrict__ bsum)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / CUT_SCAN_CHUNK];
}

// stable scatter into slab order: perm[pos] = i, rank[i] = pos, fsort[pos] = fpos[i]
__global__ void k_cut_scatter(const float4* __restrict__ fpos, int N, float zoff, float inv_w, int nslab, int nblk,
                              const int* __restrict__ boff, int* __restrict__ perm, int* __restrict__ rank,
                              float4* __restrict__ fsort)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const float4 p = i < N ? fpos[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int key = i < N ? slab_of(p.z, zoff, inv_w, nslab) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key < 0) return;
    const int pos = boff[(long long)key * nblk + (i >> 5)] + __popc(peers & ((1u << lane) - 1u));
    perm[pos] = i;
    rank[i] = pos;
    fsort[pos] = p;
}

// far-away dummies after the sorted ions (never within the cutoff of anything)
__global__ void k_cut_dummies(float4* __restrict__ fsort, int N, int n_pad)
{
    const int i = N + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const float far = 3.0e4f + 7.0f * (float)(i - N);
    fsort[i] = make_float4(far, far, far, 0.0f);
}

// bounding box of the real ions of each tile (w = 1 if the tile holds any)
__global__ void k_cut_boxes(const float4* __restrict__ fsort, int N, int TI, float4* __restrict__ lo,
                            float4* __restrict__ hi)
{
    __shared__ float s[6][32];
    const int t = blockIdx.x;
    const int q0 = t * TI, q1 = min(N, q0 + TI);
    float mn[3] = {3e38f, 3e38f, 3e38f}, mx[3] = {-3e38f, -3e38f, -3e38f};
    for (int q = q0 + (int)threadIdx.x; q < q1; q += blockDim.x) {
        const float4 p = fsort[q];
        mn[0] = fminf(mn[0], p.x), mn[1] = fminf(mn[1], p.y), mn[2] = fminf(mn[2], p.z);
        mx[0] = fmaxf(mx[0], p.x), mx[1] = fmaxf(mx[1], p.y), mx[2] = fmaxf(mx[2], p.z);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[c] = fminf(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmaxf(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
    if (lane == 0)
        for (int c = 0; c < 3; ++c) s[c][w] = mn[c], s[3 + c][w] = mx[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww)
            for (int c = 0; c < 3; ++c) s[c][0] = fminf(s[c][0], s[c][ww]), s[3 + c][0] = fmaxf(s[3 + c][0], s[3 + c][ww]);
        const float any = q1 > q0 ? 1.f : 0.f;
        lo[t] = make_float4(s[0][0], s[1][0], s[2][0], any);
        hi[t] = make_float4(s[3][0], s[4][0], s[5][0], any);
    }
}

__device__ __forceinline__ bool tiles_meet(float4 la, float4 ha, float4 lb, float4 hb, float rc2)
{
    if (la.w == 0.f || lb.w == 0.f) return false;
    const float gx = fmaxf(0.f, fmaxf(lb.x - ha.x, la.x - hb.x));
    const float gy = fmaxf(0.f, fmaxf(lb.y - ha.y, la.y - hb.y));
    const float gz = fmaxf(0.f, fmaxf(lb.z - ha.z, la.z - hb.z));
    return fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < rc2;
}

constexpr int CUT_PLAIN = 1 << 30;  // unit flag: every pair inside the switching distance

// farthest distance^2 between two boxes: below the switching distance every pair of the
// two tiles has S = 1 and S' = 0, and the plain coefficient gives the same bits
__device__ __forceinline__ float boxes_far2(float4 la, float4 ha, float4 lb, float4 hb)
{
    const float fx = fmaxf(hb.x - la.x, ha.x - lb.x), fy = fmaxf(hb.y - la.y, ha.y - lb.y);
    const float fz = fmaxf(hb.z - la.z, ha.z - lb.z);
    return fmaf(fx, fx, fmaf(fy, fy, fz * fz));
}

// Tile pairs (I, J >= I) of the tiles whose boxes come closer than the cutoff, in row
// order and ascending J within a row.  One warp per tile in both passes; T <= CUT_MAX_TILES.

// pass 1: tile pairs (J >= I) per tile
__global__ void k_cut_count(const float4* __restrict__ lo, const float4* __restrict__ hi, int T, float rc2,
                            int* __restrict__ ucnt)
{
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (I >= T) return;
    const float4 la = lo[I], ha = hi[I];
    int nu = 0;
    for (int J = I + lane; J < T; J += 32) nu += tiles_meet(la, ha, lo[J], hi[J], rc2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nu += __shfl_xor_sync(0xffffffffu, nu, o);
    if (lane == 0) ucnt[I] = nu;
}

// pass 2 (one CTA of 1024): exclusive scan of the counts, unit starts and unit count
__global__ void __launch_bounds__(1024) k_cut_offsets(const int* __restrict__ ucnt, int T, int* __restrict__ ustart,
                                                      int* __restrict__ n_units)
{
    __shared__ int s_w[32];
    constexpr int PER = CUT_MAX_TILES / 1024;
    const int base = threadIdx.x * PER;
    int u[PER], su = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        u[k] = base + k < T ? ucnt[base + k] : 0;
        su += u[k];
    }
    int tu;
    int ru = block_excl_scan(su, s_w, tu);
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (base + k < T) {
            ustart[base + k] = ru;
            ru += u[k];
        }
    if (threadIdx.x == 0) *n_units = tu;
}

// pass 3: the tile pairs (ballot prefix per group of 32) with the plain flag
__global__ void k_cut_fill(const float4* __restrict__ lo, const float4* __restrict__ hi, int T, float rc2, float rs2,
                           const int* __restrict__ ustart, int2* __restrict__ units)
{
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (I >= T) return;
    const float4 la = lo[I], ha = hi[I];
    int k = ustart[I];
    for (int J0 = I; J0 < T; J0 += 32) {
        const int J = J0 + lane;
        const bool m = J < T && tiles_meet(la, ha, lo[J], hi[J], rc2);
        const unsigned mask = __ballot_sync(0xffffffffu, m);
        if (m) {
            const bool plain = boxes_far2(la, ha, lo[J], hi[J]) < rs2;
            units[k + __popc(mask & ((1u << lane) - 1u))] = make_int2(I, J | (plain ? CUT_PLAIN : 0));
        }
        k += __popc(mask);
    }
}

// persistent CTAs over the listed tile pairs (their number is read on the device)
template <int BT, int IPT>
__global__ void __launch_bounds__(BT, (IPT == 8 ? 65536 / (BT * 128) : 1))
    k_forces_cut(const float4* __restrict__ fsort, ForceArgs F, const int2* __restrict__ units,
                 const int* __restrict__ n_units)
{
    __shared__ float s_acc[2][3][BT / 32][SYM_SUB];
    __shared__ float4 sj[BT];
    __shared__ long long s_u;
    const long long U = *n_units;
    for (;;) {
        const long long u = next_unit(F.sched, s_u);
        if (u >= U) break;
        const int2 t = units[u];  // (I, J | plain flag)
        if (t.y & CUT_PLAIN)
            sym2_unit<BT, IPT, false>(fsort, F, t.x, t.y & (CUT_PLAIN - 1), s_acc, sj);
        else
            sym2_unit<BT, IPT, true>(fsort, F, t.x, t.y, s_acc, sj);
    }
    leave_queue(F.sched);
}

static int ckc(cudaError_t e) { return e == cudaSuccess ? 0 : (int)e; }

int cut_blocks_per_sm(int ipt)
{
    int nb = 0;
    const void* fn = ipt == 4 ? (const void*)k_forces_cut<256, 4> : (const void*)k_forces_cut<64, 8>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, ipt == 4 ? 256 : 64, 0) != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

int launch_cut_dummies(const CutBufs& C, int N, int n_pad, cudaStream_t s)
{
    if (n_pad > N) k_cut_dummies<<<(n_pad - N + 255) / 256, 256, 0, s>>>(C.fsort, N, n_pad);
    return ckc(cudaGetLastError());
}

int launch_forces_cut(const Phys& P, const Bufs& B, const ForceArgs& F, const CutBufs& C, int grid, cudaStream_t s)
{
    const int N = P.N;
    if (N == 0 || (P.flags & OD_F_NO_IONION)) return 0;
    if (!F.sched) return (int)cudaErrorInvalidValue;
    const int nblk = (N + 31) / 32;
    const long long M = (long long)C.nslab * nblk;
    int rc;
    if ((rc = ckc(cudaMemsetAsync(C.bcount, 0, sizeof(int) * M, s)))) return rc;
    const int nthreads = nblk * 32;
    k_cut_hist<<<(nthreads + 255) / 256, 256, 0, s>>>(B.fpos, N, C.zoff, C.inv_w, C.nslab, nblk, C.bcount);
    const int nchunk = (int)((M + CUT_SCAN_CHUNK - 1) / CUT_SCAN_CHUNK);
    k_cut_scan_chunks<<<nchunk, 1024, 0, s>>>(C.bcount, C.boff, M, C.bsum);
    k_cut_scan_sums<<<1, 1024, 0, s>>>(C.bsum, nchunk);
    k_cut_scan_add<<<(int)((M + 255) / 256), 256, 0, s>>>(C.boff, M, C.bsum);
    k_cut_scatter<<<(nthreads + 255) / 256, 256, 0, s>>>(B.fpos, N, C.zoff, C.inv_w, C.nslab, nblk, C.boff, C.perm,
                                                        C.rank, C.fsort);
    // the padding after the sorted ions (its length changes with N)
    if (F.n_pad > N) k_cut_dummies<<<(F.n_pad - N + 255) / 256, 256, 0, s>>>(C.fsort, N, F.n_pad);
    const int T = F.n_pad / F.TI;
    k_cut_boxes<<<T, 256, 0, s>>>(C.fsort, N, F.TI, C.box_lo, C.box_hi);
    const int wb = (T + 7) / 8;  // 8 warps per CTA, one per tile
    k_cut_count<<<wb, 256, 0, s>>>(C.box_lo, C.box_hi, T, C.rc2_tile, C.ucnt);
    k_cut_offsets<<<1, 1024, 0, s>>>(C.ucnt, T, C.ustart, C.n_units);
    k_cut_fill<<<wb, 256, 0, s>>>(C.box_lo, C.box_hi, T, C.rc2_tile, C.rs2_tile, C.ustart, C.units);
    if (F.TI == 1024)
        k_forces_cut<256, 4><<<grid, 256, 0, s>>>(C.fsort, F, C.units, C.n_units);
    else  // 512-ion tiles: 64 threads x 8 targets
        k_forces_cut<64, 8><<<grid, 64, 0, s>>>(C.fsort, F, C.units, C.n_units);
    return ckc(cudaGetLastError());
}

}  // namespace od

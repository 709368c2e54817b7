// sort.cu -- depth ordering and tile binning of the projected Gaussians.
//
// Sec. III-A of 3DGS-ReLoc composites each pixel's Gaussians "sorted by
// depth".  Per view the required order of a tile's list is (depth, Gaussian
// index).  It is produced in two stable stages instead of one wide-key sort:
//   1. a stable LSD radix sort of the visible (view, Gaussian) pairs by the
//      float32 depth bit pattern (4 passes of 8 bits; the first pass also
//      drops invisible pairs, so compaction costs nothing extra);
//   2. emission of one (tile, Gaussian) entry per covered tile in that depth
//      order (K3), then a stable LSD radix sort by tile id (K4, 1-2 passes).
// Stability of both stages makes every tile's list ordered by depth and, for
// equal depth bits, by Gaussian index -- the same order as one stable sort of
// view|tile|depth keys emitted in index order, with far fewer passes over the
// (much larger) instance list.
//
// Every per-view array sits at a host-planned offset with a host-planned
// capacity, and chunk tables map a block to its view and chunk, so valid
// lengths stay in device memory: no host round trip between stages.
#include "internal.cuh"

namespace reloc {

static_assert(SORT_THREADS == RADIX, "scatter assigns one digit per thread");

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Block-wide exclusive scan of one value per thread; *total gets the sum.
// s_tmp: 33 words of shared memory.  All threads must call it.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t *s_tmp, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_tmp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? s_tmp[lane] : 0u, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        s_tmp[lane] = wi - w;
        if (lane == 31) s_tmp[32] = wi;
    }
    __syncthreads();
    uint32_t r = s_tmp[warp] + inc - x;
    *total = s_tmp[32];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------ upsweep ------
// Per chunk digit counts -> hist[s][d][k] (digit-major inside a segment, so
// one exclusive scan of the segment's block gives every chunk's offsets).
__global__ void __launch_bounds__(SORT_THREADS) k_radix_upsweep(RadixPass p)
{
    __shared__ uint32_t s_h[RADIX];
    const int c = blockIdx.x;
    const int s = find_segment(p.chunk_base, p.n_seg, c);
    const int k = c - p.chunk_base[s], cps = p.chunk_base[s + 1] - p.chunk_base[s];
    s_h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t cap = p.seg_off[s + 1] - p.seg_off[s];
    const int64_t seg_len = p.len ? min64(p.len[s], cap) : cap;
    const int64_t begin = (int64_t)k * SORT_CHUNK;
    const int n = (int)max64(0, min64(SORT_CHUNK, seg_len - begin));
    const int64_t base = p.seg_off[s] + begin;
    const unsigned lt = lanemask_lt();
    for (int b = 0; b < n; b += SORT_THREADS) {
        const int idx = b + threadIdx.x;
        bool valid = idx < n;
        uint32_t d = RADIX;
        if (valid) {
            if (p.filt) valid = p.filt[base + idx] != 0;
            if (valid) d = (p.keys_in[base + idx] >> p.shift) & p.mask;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lt) == 0) atomicAdd(&s_h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    p.hist[(int64_t)RADIX * p.chunk_base[s] + (int64_t)threadIdx.x * cps + k] = s_h[threadIdx.x];
}

// --------------------------------------------------- segment scan ----------
// In-place exclusive scan of `count` words per segment; total_out[s] = sum.
// In-place exclusive scan of segment s = data[mult*base[s], mult*base[s+1]);
// total_out[s] = its sum.  One block per segment walks it in tiles of
// SCAN_THREADS * 4 words (each thread 4 consecutive words, coalesced),
// carrying the running total from tile to tile.
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_IPT = 4;
__global__ void __launch_bounds__(SCAN_THREADS)
k_seg_scan(uint32_t *data, const int32_t *__restrict__ base, int mult, uint32_t *total_out)
{
    __shared__ uint32_t s_tmp[33];
    uint32_t *a = data + (int64_t)mult * base[blockIdx.x];
    const int64_t count = (int64_t)mult * (base[blockIdx.x + 1] - base[blockIdx.x]);
    uint32_t carry = 0;
    for (int64_t t0 = 0; t0 < count; t0 += SCAN_THREADS * SCAN_IPT) {
        const int64_t i0 = t0 + (int64_t)threadIdx.x * SCAN_IPT;
        uint32_t v[SCAN_IPT], sum = 0;
#pragma unroll
        for (int j = 0; j < SCAN_IPT; ++j) {
            v[j] = i0 + j < count ? a[i0 + j] : 0u;
            sum += v[j];
        }
        uint32_t tot;
        uint32_t run = carry + block_excl_scan(sum, s_tmp, &tot);
#pragma unroll
        for (int j = 0; j < SCAN_IPT; ++j) {
            if (i0 + j < count) a[i0 + j] = run;
            run += v[j];
        }
        carry += tot;
    }
    if (total_out && threadIdx.x == 0) total_out[blockIdx.x] = carry;
}

// ------------------------------------------------------------ scatter ------
// Stable scatter of one chunk.  Warp w owns the contiguous items
// [w*512, (w+1)*512) and ranks them round by round with __match_any_sync, so
// ranks follow input order; per-warp digit counters then give each warp's
// offset inside the block.  Items are staged digit-sorted in shared memory
// and written out in runs (coalesced).
__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(RadixPass p)
{
    constexpr int NW = SORT_THREADS / 32;
    __shared__ uint32_t s_wcnt[NW][RADIX];
    __shared__ uint32_t s_boff[RADIX];
    __shared__ uint32_t s_goff[RADIX];
    __shared__ uint32_t s_key[SORT_CHUNK];
    __shared__ uint32_t s_val[SORT_CHUNK];
    __shared__ uint32_t s_tmp[33];

    const int c = blockIdx.x;
    const int s = find_segment(p.chunk_base, p.n_seg, c);
    const int k = c - p.chunk_base[s], cps = p.chunk_base[s + 1] - p.chunk_base[s];
    const int64_t cap = p.seg_off[s + 1] - p.seg_off[s];
    const int64_t seg_len = p.len ? min64(p.len[s], cap) : cap;
    const int64_t begin = (int64_t)k * SORT_CHUNK;
    if (begin >= seg_len) return;                       // uniform for the block
    const int n = (int)min64(SORT_CHUNK, seg_len - begin);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 0; w < NW; ++w) s_wcnt[w][threadIdx.x] = 0;
    __syncthreads();

    const int64_t base = p.seg_off[s] + begin;
    const unsigned lt = lanemask_lt();
    uint32_t key[SORT_IPT], val[SORT_IPT], rank[SORT_IPT];
#pragma unroll
    for (int r = 0; r < SORT_IPT; ++r) {
        const int idx = warp * (32 * SORT_IPT) + r * 32 + lane;
        bool valid = idx < n;
        uint32_t kk = 0, vv = 0;
        if (valid) {
            if (p.filt) valid = p.filt[base + idx] != 0;
            kk = p.keys_in[base + idx];
            vv = p.vals_in ? p.vals_in[base + idx] : (uint32_t)(begin + idx);
        }
        const uint32_t d = valid ? (kk >> p.shift) & p.mask : (uint32_t)RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (valid) before = s_wcnt[warp][d];
        __syncwarp();
        if (valid && (peers & lt) == 0) s_wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
        key[r] = kk;
        val[r] = vv;
        rank[r] = valid ? before + __popc(peers & lt) : 0xFFFFFFFFu;
    }
    __syncthreads();
    // thread d: prefix of digit d over warps, then block scan over digits
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        uint32_t t = s_wcnt[w][threadIdx.x];
        s_wcnt[w][threadIdx.x] = tot;
        tot += t;
    }
    uint32_t nvalid;
    const uint32_t excl = block_excl_scan(tot, s_tmp, &nvalid);
    s_boff[threadIdx.x] = excl;
    s_goff[threadIdx.x] = p.hist[(int64_t)RADIX * p.chunk_base[s] + (int64_t)threadIdx.x * cps + k];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SORT_IPT; ++r) {
        if (rank[r] != 0xFFFFFFFFu) {
            const uint32_t d = (key[r] >> p.shift) & p.mask;
            const uint32_t pos = s_boff[d] + s_wcnt[warp][d] + rank[r];
            s_key[pos] = key[r];
            s_val[pos] = val[r];
        }
    }
    __syncthreads();
    const int64_t obase = p.seg_off[s];
    for (int j = threadIdx.x; j < (int)nvalid; j += SORT_THREADS) {
        const uint32_t kk = s_key[j];
        const uint32_t d = (kk >> p.shift) & p.mask;
        const int64_t pos = obase + s_goff[d] + (uint32_t)(j - s_boff[d]);
        p.keys_out[pos] = kk;
        p.vals_out[pos] = s_val[j];
    }
}

cudaError_t launch_radix_pass(const RadixPass &p, cudaStream_t st)
{
    if (p.n_seg <= 0 || p.total_chunks <= 0) return cudaSuccess;
    k_radix_upsweep<<<p.total_chunks, SORT_THREADS, 0, st>>>(p);
    k_seg_scan<<<p.n_seg, SCAN_THREADS, 0, st>>>(p.hist, p.chunk_base, RADIX, p.len_out);
    k_radix_scatter<<<p.total_chunks, SORT_THREADS, 0, st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------- K3 emit -----

__global__ void __launch_bounds__(EMIT_THREADS)
k_emit_sums(const uint32_t *__restrict__ sorted_g, const uint32_t *__restrict__ n_vis,
            const uint32_t *__restrict__ ntiles, Layout L, uint32_t *__restrict__ chunk_sums)
{
    __shared__ uint32_t s_tmp[33];
    const int c = blockIdx.x;
    const int v = find_segment(L.ce_base, L.V, c);
    const int k = c - L.ce_base[v];
    const int64_t S = L.vd_off[v + 1] - L.vd_off[v];
    const int64_t nv = min64(n_vis[v], S);
    const int64_t begin = (int64_t)k * EMIT_CHUNK;
    const int n = (int)max64(0, min64(EMIT_CHUNK, nv - begin));
    const uint32_t *g = sorted_g + L.vd_off[v] + begin;
    const uint32_t *nt = ntiles + L.vd_off[v];
    uint32_t sum = 0;
    for (int j = threadIdx.x; j < n; j += EMIT_THREADS) sum += nt[g[j]];
    uint32_t tot;
    block_excl_scan(sum, s_tmp, &tot);
    if (threadIdx.x == 0) chunk_sums[c] = tot;
}

__global__ void __launch_bounds__(EMIT_THREADS)
k_emit(const uint32_t *__restrict__ sorted_g, const uint32_t *__restrict__ n_vis,
       const uint32_t *__restrict__ ntiles, const uint2 *__restrict__ rect, Layout L, int ntx,
       const uint32_t *__restrict__ chunk_off, const uint32_t *__restrict__ n_inst,
       uint32_t *__restrict__ inst_tile, uint32_t *__restrict__ inst_gauss, int *overflow)
{
    __shared__ uint32_t s_g[EMIT_CHUNK];
    __shared__ uint32_t s_off[EMIT_CHUNK];
    __shared__ uint2 s_rect[EMIT_CHUNK];
    __shared__ uint2 s_win[EMIT_WINDOW];
    __shared__ uint32_t s_tmp[33];
    const int c = blockIdx.x;
    const int v = find_segment(L.ce_base, L.V, c);
    const int k = c - L.ce_base[v];
    const int64_t cap = L.io_off[v + 1] - L.io_off[v];
    if ((int64_t)n_inst[v] > cap) {                     // this view does not fit
        if (k == 0 && threadIdx.x == 0) atomicExch(overflow, 1);
        return;
    }
    const int64_t S = L.vd_off[v + 1] - L.vd_off[v];
    const int64_t nv = min64(n_vis[v], S);
    const int64_t begin = (int64_t)k * EMIT_CHUNK;
    if (begin >= nv) return;
    const int n = (int)min64(EMIT_CHUNK, nv - begin);
    const uint32_t *g = sorted_g + L.vd_off[v] + begin;
    for (int j = threadIdx.x; j < n; j += EMIT_THREADS) {
        const uint32_t gi = g[j];
        s_g[j] = gi;
        s_off[j] = ntiles[L.vd_off[v] + gi];
        s_rect[j] = rect[L.vd_off[v] + gi];
    }
    __syncthreads();
    // blocked exclusive scan of the counts (item order = depth order)
    const int j0 = threadIdx.x * EMIT_IPT;
    uint32_t loc[EMIT_IPT];
    uint32_t sum = 0;
#pragma unroll
    for (int r = 0; r < EMIT_IPT; ++r) {
        const int j = j0 + r;
        loc[r] = j < n ? s_off[j] : 0u;
        sum += loc[r];
    }
    uint32_t total;
    uint32_t run = block_excl_scan(sum, s_tmp, &total);
#pragma unroll
    for (int r = 0; r < EMIT_IPT; ++r) {
        const int j = j0 + r;
        if (j < n) s_off[j] = run;
        run += loc[r];
    }
    __syncthreads();
    // Windows of EMIT_THREADS * EMIT_RUN entries: each thread fills EMIT_RUN
    // consecutive entries of the window in shared memory (one binary search,
    // then a walk along the items' tile rectangles, row-major), and the block
    // copies the window out with coalesced stores.
    const int64_t obase = L.io_off[v] + chunk_off[c];
    for (uint32_t w0 = 0; w0 < total; w0 += EMIT_WINDOW) {
        const uint32_t m0 = w0 + threadIdx.x * EMIT_RUN;
        if (m0 < total) {
            int lo = 0, hi = n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= m0) lo = mid; else hi = mid - 1;
            }
            uint2 rc = s_rect[lo];
            uint32_t x0 = rc.x & 0xFFFFu, x1 = rc.x >> 16, y0 = rc.y & 0xFFFFu;
            const uint32_t local = m0 - s_off[lo], w = x1 - x0 + 1;
            uint32_t ty = y0 + local / w, tx = x0 + local % w;
            uint32_t end = lo + 1 < n ? s_off[lo + 1] : total;
            uint32_t gi = s_g[lo];
            const uint32_t m1 = min(total, m0 + EMIT_RUN);
            for (uint32_t m = m0; m < m1; ++m) {
                while (m == end) {                   // next item with tiles
                    ++lo;
                    rc = s_rect[lo];
                    x0 = rc.x & 0xFFFFu; x1 = rc.x >> 16; y0 = rc.y & 0xFFFFu;
                    tx = x0;
                    ty = y0;
                    gi = s_g[lo];
                    end = lo + 1 < n ? s_off[lo + 1] : total;
                }
                s_win[m - w0] = make_uint2(ty * (uint32_t)ntx + tx, gi);
                if (++tx > x1) { tx = x0; ++ty; }
            }
        }
        __syncthreads();
        const uint32_t wn = min((uint32_t)EMIT_WINDOW, total - w0);
        for (uint32_t j = threadIdx.x; j < wn; j += EMIT_THREADS) {
            const uint2 e = s_win[j];
            inst_tile[obase + w0 + j] = e.x;
            inst_gauss[obase + w0 + j] = e.y;
        }
        __syncthreads();
    }
}

cudaError_t launch_emit(const uint32_t *sorted_g, const uint32_t *n_vis, const uint32_t *ntiles, const uint2 *rect,
                        const Layout &L, int n_chunks, int ntx, uint32_t *chunk_sums, uint32_t *inst_tile,
                        uint32_t *inst_gauss, uint32_t *n_inst, int *overflow, cudaStream_t st)
{
    if (n_chunks <= 0 || L.V <= 0) return cudaSuccess;
    k_emit_sums<<<n_chunks, EMIT_THREADS, 0, st>>>(sorted_g, n_vis, ntiles, L, chunk_sums);
    k_seg_scan<<<L.V, SCAN_THREADS, 0, st>>>(chunk_sums, L.ce_base, 1, n_inst);
    k_emit<<<n_chunks, EMIT_THREADS, 0, st>>>(sorted_g, n_vis, ntiles, rect, L, ntx, chunk_sums, n_inst, inst_tile,
                                              inst_gauss, overflow);
    return cudaGetLastError();
}

// ------------------------------------------------------------ K5 ranges ----

__global__ void k_ranges(const uint32_t *__restrict__ tiles, const uint32_t *__restrict__ n_inst, Layout L,
                         int n_tiles, int2 *__restrict__ ranges, const int *__restrict__ overflow)
{
    if (*overflow) return;
    const int v = blockIdx.y;
    const int64_t n = min64(n_inst[v], L.io_off[v + 1] - L.io_off[v]);
    const uint32_t *t = tiles + L.io_off[v];
    int2 *R = ranges + (int64_t)v * n_tiles;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t tj = t[j];
        if (j == 0 || t[j - 1] != tj) R[tj].x = (int)j;
        if (j == n - 1 || t[j + 1] != tj) R[tj].y = (int)(j + 1);
    }
}

cudaError_t launch_ranges(const uint32_t *inst_tile, const uint32_t *n_inst, const Layout &L, int n_tiles,
                          int2 *ranges, const int *overflow, cudaStream_t st)
{
    if (L.V <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(int2) * (size_t)L.V * n_tiles, st);
    if (e != cudaSuccess) return e;
    dim3 grid(64, L.V);
    k_ranges<<<grid, 256, 0, st>>>(inst_tile, n_inst, L, n_tiles, ranges, overflow);
    return cudaGetLastError();
}

}  // namespace reloc

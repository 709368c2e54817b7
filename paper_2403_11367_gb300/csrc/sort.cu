// sort.cu -- depth ordering and tile binning of the projected Gaussians.
//
// Sec. III-A of 3DGS-ReLoc composites each pixel's Gaussians "sorted by
// depth".  Per view the required order of a tile's list is (depth, Gaussian
// index).  It is produced without any sort over the (much larger) instance
// list:
//   1. a stable LSD radix sort of the visible (view, Gaussian) pairs by the
//      float32 depth bit pattern (4 passes of 8 bits; the first pass also
//      drops invisible pairs, so compaction costs nothing extra);
//   2. per chunk of that depth order, tile coverage counts (K3: 2D difference
//      arrays), scanned into each tile's list start and each chunk's slot in it;
//   3. emission of every (tile, Gaussian) instance straight into its slot, a
//      warp per (chunk, tile row) walking the chunk in depth order (K4).
// Stability of the depth sort makes every tile's list ordered by depth and,
// for equal depth bits, by Gaussian index -- the same order as one stable sort
// of view|tile|depth keys emitted in index order.
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
// Each key adds 1 to its warp's own histogram with a shared-memory atomic;
// the warps' histograms are summed at the end.  (Merging a warp's equal
// digits first with __match_any_sync, one atomic per distinct digit, kept
// the MIO queue full: the depth sort took 0.66 instead of 0.51 ms per
// 64-candidate query, on the exponent byte too, where few values recur.)
__global__ void __launch_bounds__(SORT_THREADS) k_radix_upsweep(RadixPass p)
{
    constexpr int NW = SORT_THREADS / 32;
    __shared__ uint32_t s_h[NW][RADIX];
    const int c = blockIdx.x;
    const int s = find_segment(p.chunk_base, p.n_seg, c);
    const int k = c - p.chunk_base[s], cps = p.chunk_base[s + 1] - p.chunk_base[s];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int w = 0; w < NW; ++w) s_h[w][threadIdx.x] = 0;
    __syncthreads();
    const int64_t cap = p.seg_off[s + 1] - p.seg_off[s];
    const int64_t seg_len = p.len ? min64(p.len[s], cap) : cap;
    const int64_t begin = (int64_t)k * SORT_CHUNK;
    const int n = (int)max64(0, min64(SORT_CHUNK, seg_len - begin));
    const int64_t base = p.seg_off[s] + begin;
    // all of this thread's loads first (independent, in flight together), then the counts
    uint32_t d[SORT_IPT];
#pragma unroll
    for (int r = 0; r < SORT_IPT; ++r) {
        const int idx = r * SORT_THREADS + threadIdx.x;
        d[r] = RADIX;
        if (idx < n) {
            const uint32_t k = p.keys_in[base + idx];
            const bool keep = !p.drop_culled || k != 0xFFFFFFFFu;
            d[r] = keep ? (k >> p.shift) & p.mask : (uint32_t)RADIX;
        }
    }
#pragma unroll
    for (int r = 0; r < SORT_IPT; ++r)
        if (d[r] != (uint32_t)RADIX) atomicAdd(&s_h[warp][d[r]], 1u);
    __syncthreads();
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) cnt += s_h[w][threadIdx.x];
    p.hist[(int64_t)RADIX * p.chunk_base[s] + (int64_t)threadIdx.x * cps + k] = cnt;
    if (cnt) atomicAdd(p.dtot + (int64_t)RADIX * s + threadIdx.x, cnt);
}

// ------------------------------------------------------- digit offsets -----
// Exclusive offsets of one pass in place: the segment's counts are stored
// digit-major ([digit][chunk]), so the offset of (d, k) is the total of all
// smaller digits (dtot, summed by the upsweep) plus the counts of digit d in
// the chunks before k.  A warp per (segment, digit) takes the first from
// dtot and scans the second 32 chunks at a time; len_out[s] (may be null) =
// the segment's total.
constexpr int DSCAN_WARPS = 8;
__global__ void __launch_bounds__(32 * DSCAN_WARPS)
k_digit_scan(uint32_t *hist, const uint32_t *__restrict__ dtot, const int32_t *__restrict__ chunk_base,
             uint32_t *len_out)
{
    const int s = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = blockIdx.y * DSCAN_WARPS + warp;
    const uint32_t *dt = dtot + (int64_t)RADIX * s;
    uint32_t below = 0, all = 0;
    for (int i = lane; i < RADIX; i += 32) {
        const uint32_t x = dt[i];
        below += i < d ? x : 0u;
        all += x;
    }
    below = __reduce_add_sync(0xffffffffu, below);
    all = __reduce_add_sync(0xffffffffu, all);
    if (len_out && d == 0 && lane == 0) len_out[s] = all;
    const int cps = chunk_base[s + 1] - chunk_base[s];
    uint32_t *h = hist + (int64_t)RADIX * chunk_base[s] + (int64_t)d * cps;
    uint32_t carry = below;
    for (int k0 = 0; k0 < cps; k0 += 32) {
        const int k = k0 + lane;
        const uint32_t x = k < cps ? h[k] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (k < cps) h[k] = carry + inc - x;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
}

// ------------------------------------------------------------ scatter ------
// Stable scatter of one chunk.  Warp w owns the contiguous items
// [w*256, (w+1)*256) and ranks them round by round (the lanes sharing a
// digit from nine ballots, one per bit of the digit), so ranks follow input
// order; per-warp digit counters then give each warp's offset inside the
// block.  Items are staged digit-sorted in shared memory and written out in
// runs (coalesced).
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
    bool vld[SORT_IPT];
    // all of this thread's loads first (independent, in flight together), then the ranks
#pragma unroll
    for (int r = 0; r < SORT_IPT; ++r) {
        const int idx = warp * (32 * SORT_IPT) + r * 32 + lane;
        vld[r] = idx < n;
        key[r] = 0u;
        val[r] = 0u;
        if (vld[r]) {
            key[r] = p.keys_in[base + idx];
            val[r] = p.vals_in ? p.vals_in[base + idx] : (uint32_t)(begin + idx);
            if (p.drop_culled) vld[r] = key[r] != 0xFFFFFFFFu;
        }
    }
#pragma unroll
    for (int r = 0; r < SORT_IPT; ++r) {
        const bool valid = vld[r];
        const uint32_t kk = key[r], vv = val[r];
        const uint32_t d = valid ? (kk >> p.shift) & p.mask : (uint32_t)RADIX;
        // lanes holding the same digit (or both invalid): the intersection of
        // nine ballots, one per bit of d (0..RADIX)
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const bool set = ((d >> b) & 1u) != 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, set);
            peers &= set ? bal : ~bal;
        }
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
    k_digit_scan<<<dim3(p.n_seg, RADIX / DSCAN_WARPS), 32 * DSCAN_WARPS, 0, st>>>(p.hist, p.dtot, p.chunk_base,
                                                                                   p.len_out);
    k_radix_scatter<<<p.total_chunks, SORT_THREADS, 0, st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------ K3 tile counts -----
// Each view's visible Gaussians, in depth order, are cut into chunks of
// cp.bin_chunk.  Per chunk, k_tile_count counts how many of them cover each
// tile: every rectangle adds +1/-1 at its four corners of a 2D difference
// array in shared memory, and two prefix sums (along x, then y) turn it into
// counts.  The tile grid is processed in row bands that fit shared memory.
// It also writes the rectangles in depth order (srect) for K4.
constexpr int BIN_THREADS = 256;

__global__ void __launch_bounds__(BIN_THREADS)
k_tile_count(const uint32_t *__restrict__ sorted_g, const uint32_t *__restrict__ n_vis,
             const uint2 *__restrict__ rect, Layout L, CamParams cp, int band_rows, uint2 *__restrict__ srect,
             uint32_t *__restrict__ bhist)
{
    extern __shared__ uint32_t s_d[];   // (band_rows + 1) x (ntx + 1)
    const int c = blockIdx.x;
    const int v = find_segment(L.cb_base, L.V, c);
    const int k = c - L.cb_base[v];
    const int64_t S = L.vd_off[v + 1] - L.vd_off[v];
    const int64_t nv = min64(n_vis[v], S);
    const int64_t begin = (int64_t)k * cp.bin_chunk;
    if (begin >= nv) return;
    const int n = (int)min64(cp.bin_chunk, nv - begin);
    const int ntx = cp.ntx, W = ntx + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t *g = sorted_g + L.vd_off[v] + begin;
    const uint2 *rv = rect + L.vd_off[v];
    uint2 *sr = srect + L.vd_off[v] + begin;
    uint32_t *h = bhist + (int64_t)cp.n_tiles * c;
    for (int r0 = 0; r0 < cp.nty; r0 += band_rows) {
        const int r1 = min(cp.nty, r0 + band_rows), H = r1 - r0;
        for (int i = threadIdx.x; i < (H + 1) * W; i += BIN_THREADS) s_d[i] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += BIN_THREADS) {
            uint2 rc;
            if (r0 == 0) {               // first band: gather in depth order
                rc = rv[g[j]];
                sr[j] = rc;
            } else {
                rc = sr[j];              // written by this thread in band 0
            }
            const int y0 = (int)(rc.y & 0xFFFFu), y1 = (int)(rc.y >> 16);
            if (y1 < r0 || y0 >= r1) continue;
            const int x0 = (int)(rc.x & 0xFFFFu), x1 = (int)(rc.x >> 16);
            const int ya = max(y0, r0) - r0, yb = min(y1, r1 - 1) - r0 + 1;
            atomicAdd(&s_d[ya * W + x0], 1u);
            atomicAdd(&s_d[ya * W + x1 + 1], 0xFFFFFFFFu);
            atomicAdd(&s_d[yb * W + x0], 0xFFFFFFFFu);
            atomicAdd(&s_d[yb * W + x1 + 1], 1u);
        }
        __syncthreads();
        for (int y = warp; y < H; y += BIN_THREADS / 32) {      // prefix along x: a warp per row
            uint32_t carry = 0;
            for (int x0 = 0; x0 < ntx; x0 += 32) {
                const int x = x0 + lane;
                uint32_t inc = x < ntx ? s_d[y * W + x] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t;
                }
                if (x < ntx) s_d[y * W + x] = carry + inc;
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        __syncthreads();
        for (int x = threadIdx.x; x < ntx; x += BIN_THREADS) {  // prefix along y: a thread per column
            uint32_t run = 0;
            for (int y = 0; y < H; ++y) {
                run += s_d[y * W + x];
                s_d[y * W + x] = run;
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < H * ntx; t += BIN_THREADS) {
            const int y = t / ntx, x = t - y * ntx;
            h[(int64_t)r0 * ntx + t] = s_d[y * W + x];
        }
        __syncthreads();
    }
}

// Per view: bhist[chunk][tile] becomes the exclusive prefix over the view's
// chunks (each chunk's first slot inside a tile's list, relative to the
// tile's start), totals -> ranges[v][tile].y; then a block per view scans
// the totals in tile order into ranges[v][tile] = [begin, end) (empty tiles
// [0, 0)) and n_inst[v].  The chunk prefix: a block per (view, 32 tiles),
// eight threads per tile, each holding up to TCOL_SEG of the tile's chunks in
// registers (all its loads in flight at once), so a view's ~80 chunks are
// scanned as eight short runs plus a prefix over the eight run totals.
constexpr int TCOL_TILES = 32;
constexpr int TCOL_SEGS = 8;
constexpr int TCOL_THREADS = TCOL_TILES * TCOL_SEGS;
constexpr int TCOL_SEG = 16;                         // chunks per run in registers
constexpr int TSCAN_THREADS = 1024;

__global__ void __launch_bounds__(TCOL_THREADS, 4)
k_tile_chunk_scan(const uint32_t *__restrict__ n_vis, Layout L, CamParams cp, uint32_t *__restrict__ bhist,
                  int2 *__restrict__ ranges)
{
    __shared__ uint32_t s_run[TCOL_SEGS][TCOL_TILES];
    const int v = blockIdx.y;
    const int tl = threadIdx.x % TCOL_TILES, sg = threadIdx.x / TCOL_TILES;
    const int t = blockIdx.x * TCOL_TILES + tl;
    const int nt = cp.n_tiles;
    const int64_t S = L.vd_off[v + 1] - L.vd_off[v];
    const int64_t nv = min64(n_vis[v], S);
    const int nch = (int)ceil_div(nv, cp.bin_chunk);
    uint32_t *h = bhist + (int64_t)nt * L.cb_base[v] + t;
    const int per = (int)ceil_div(nch, TCOL_SEGS);      // chunks of this thread's run
    const int c0 = sg * per, c1 = min(nch, c0 + per);
    uint32_t sum = 0;
    if (per <= TCOL_SEG) {                              // uniform over the block
        uint32_t x[TCOL_SEG];
        uint32_t *hp = h + (int64_t)c0 * nt;
        const int m = t < nt ? c1 - c0 : 0;
#pragma unroll
        for (int j = 0; j < TCOL_SEG; ++j) x[j] = j < m ? hp[(int64_t)j * nt] : 0u;
#pragma unroll
        for (int j = 0; j < TCOL_SEG; ++j) sum += x[j];
        s_run[sg][tl] = sum;
        __syncthreads();
        if (t >= nt) return;
        uint32_t run = 0;
        for (int k = 0; k < sg; ++k) run += s_run[k][tl];
#pragma unroll
        for (int j = 0; j < TCOL_SEG; ++j)
            if (j < m) {
                hp[(int64_t)j * nt] = run;
                run += x[j];
            }
        if (sg == TCOL_SEGS - 1) ranges[(int64_t)v * nt + t].y = (int)run;
        return;
    }
    // long views (more than TCOL_SEGS * TCOL_SEG chunks) or tiles past the
    // grid: runs summed first, then rewritten
    if (t < nt)
        for (int c = c0; c < c1; ++c) sum += h[(int64_t)c * nt];
    s_run[sg][tl] = sum;
    __syncthreads();
    if (t >= nt) return;
    uint32_t run = 0;
    for (int k = 0; k < sg; ++k) run += s_run[k][tl];
    for (int c = c0; c < c1; ++c) {
        const uint32_t x = h[(int64_t)c * nt];
        h[(int64_t)c * nt] = run;
        run += x;
    }
    if (sg == TCOL_SEGS - 1) ranges[(int64_t)v * nt + t].y = (int)run;
}

__global__ void __launch_bounds__(TSCAN_THREADS)
k_tile_scan(Layout L, CamParams cp, int2 *__restrict__ ranges, uint32_t *__restrict__ n_inst, int *overflow)
{
    __shared__ uint32_t s_tmp[33];
    const int v = blockIdx.x;
    const int nt = cp.n_tiles;
    int2 *R = ranges + (int64_t)v * nt;
    uint32_t carry = 0;
    for (int t0 = 0; t0 < nt; t0 += TSCAN_THREADS) {
        const int t = t0 + threadIdx.x;
        const uint32_t x = t < nt ? (uint32_t)R[t].y : 0u;
        uint32_t tot;
        const uint32_t start = carry + block_excl_scan(x, s_tmp, &tot);
        if (t < nt) R[t] = x ? make_int2((int)start, (int)(start + x)) : make_int2(0, 0);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        n_inst[v] = carry;
        if ((int64_t)carry > L.io_off[v + 1] - L.io_off[v]) atomicExch(overflow, 1);
    }
}

cudaError_t launch_tile_count(const uint32_t *sorted_g, const uint32_t *n_vis, const uint2 *rect, const Layout &L,
                              const CamParams &cp, int n_chunks, uint2 *srect, uint32_t *bhist, int2 *ranges,
                              uint32_t *n_inst, int *overflow, cudaStream_t st)
{
    if (L.V <= 0) return cudaSuccess;
    if (n_chunks > 0) {
        const int W = cp.ntx + 1;
        const int band_rows = max(1, min(cp.nty, TILE_COUNT_SMEM / (4 * W) - 1));
        const size_t smem = 4 * (size_t)(band_rows + 1) * W;
        k_tile_count<<<n_chunks, BIN_THREADS, smem, st>>>(sorted_g, n_vis, rect, L, cp, band_rows, srect, bhist);
    }
    k_tile_chunk_scan<<<dim3((unsigned)ceil_div(cp.n_tiles, TCOL_TILES), L.V), TCOL_THREADS, 0, st>>>(
        n_vis, L, cp, bhist, ranges);
    k_tile_scan<<<L.V, TSCAN_THREADS, 0, st>>>(L, cp, ranges, n_inst, overflow);
    return cudaGetLastError();
}

// ------------------------------------------------------ K4 tile emission ----
// A warp per (chunk, tile row).  The block stages the chunk's depth-ordered
// (rectangle, Gaussian) pairs in shared memory; each warp picks, in order,
// the pairs whose rectangle covers its row (ballot + popc into a per-warp
// queue of (Gaussian, column span) entries) and writes every queued pair into
// each covered tile's list at that tile's running slot.  The pairs are taken
// in depth order, so every list comes out ordered by (depth, index) without a
// sort over the instances.
//
// k_tile_emit_flat: rows of at most EMIT_FLAT_MAX_NTX tiles.  32 queued pairs
// are written at a time with no loop over tiles or column bands: queued pair
// e (lane e) XORs its lane bit into a difference array along the row at x0
// and at x1 + 1, so the array's inclusive XOR prefix is, for every tile x,
// the mask M[x] of the queued pairs covering x.  Pair e's slot in tile x is
// cnt[x] + popc(M[x] & bits below e) -- its rank among the chunk's pairs
// covering x, in depth order -- so the instances can be written in any order
// (lane e writes its pair's first EMIT_JCAP columns; the columns of wider
// spans are spread over the lanes), and then cnt[x] += popc(M[x]).
// k_tile_emit_smem: any row width, slots in shared memory, a lane per
// column of each queued pair.
constexpr int EMIT_STAGE = BIN_CHUNK_MIN;             // a whole chunk of the usual size: one barrier
constexpr int EMIT_FLAT_MAX_NTX = 256;
constexpr int EMIT_Q = 256;                           // queue ring entries per warp (>= 31 + 128)
constexpr int EMIT_JCAP = 4;                          // columns a pair's own lane writes
constexpr int EMIT_DYN_MIN_CHUNKS = 1024;             // about a full wave of eight-warp blocks

struct EmitChunk {
    int v, n;
    int64_t begin, nv;
    bool skip;
};

__device__ __forceinline__ EmitChunk emit_chunk(const uint32_t *n_vis, const uint32_t *n_inst, const Layout &L,
                                                const CamParams &cp)
{
    EmitChunk ch;
    const int c = blockIdx.x;
    ch.v = find_segment(L.cb_base, L.V, c);
    const int k = c - L.cb_base[ch.v];
    const int64_t S = L.vd_off[ch.v + 1] - L.vd_off[ch.v];
    const int64_t nv = min64(n_vis[ch.v], S);
    ch.nv = nv;
    ch.begin = (int64_t)k * cp.bin_chunk;
    ch.skip = ch.begin >= nv ||                                             // past the visible list
              (int64_t)n_inst[ch.v] > L.io_off[ch.v + 1] - L.io_off[ch.v];   // overflow: nothing emitted
    ch.n = ch.skip ? 0 : (int)min64(cp.bin_chunk, nv - ch.begin);
    return ch;
}

// RMASK (grids of at most 32 tile rows): each staged pair carries the bit
// mask of the rows its rectangle covers, so a warp's row test is one AND.
// DYN (with RMASK, chunks of at most one stage): one block per chunk, whose
// warps take the chunk's rows from a counter, heaviest row first (the row
// through the horizon holds several times the average row's instances, and
// a block of fixed rows lives as long as its heaviest one).  Otherwise a
// block per (chunk, 8 rows), a warp per row.
template <int CPL, bool RMASK, bool DYN>
__global__ void __launch_bounds__(TILE_EMIT_WARPS * 32, 6)
k_tile_emit_flat(const uint32_t *__restrict__ sorted_g, const uint2 *__restrict__ srect,
                 const uint32_t *__restrict__ n_vis, const uint32_t *__restrict__ n_inst,
                 const uint32_t *__restrict__ bhist, const int2 *__restrict__ ranges, Layout L, CamParams cp,
                 uint32_t *__restrict__ inst_gauss)
{
    static_assert(CPL % 4 == 0, "columns per lane in 16-byte groups");
    static_assert(!DYN || RMASK, "dynamic rows need the 32-row mask");
    constexpr int NC = 32 * CPL;                        // columns a warp's arrays hold (>= ntx)
    __shared__ uint32_t s_y[EMIT_STAGE];                // row mask (RMASK) or y0 | y1 << 16
    __shared__ uint32_t s_x[EMIT_STAGE];                // x0 | x1 << 16
    __shared__ uint32_t s_g[EMIT_STAGE];
    __shared__ uint16_t s_q[TILE_EMIT_WARPS][EMIT_Q];   // ring of staged-pair indices
    __shared__ __align__(16) uint32_t s_cnt[TILE_EMIT_WARPS][NC];
    __shared__ __align__(16) uint32_t s_m[TILE_EMIT_WARPS][NC + 4];   // x1 + 1 <= ntx <= NC
    __shared__ uint32_t s_load[32];                     // DYN: the chunk's instances per row
    __shared__ int s_order[32];                         // DYN: rows, heaviest first
    __shared__ int s_next;
    const EmitChunk ch = emit_chunk(n_vis, n_inst, L, cp);
    if (ch.skip) return;
    const int v = ch.v, n = ch.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ntx = cp.ntx;
    uint16_t *q = s_q[warp];
    uint32_t *out = inst_gauss + L.io_off[v];
    uint32_t *cnt = s_cnt[warp];
    uint32_t *M = s_m[warp];
    const uint32_t *hc = bhist + (int64_t)cp.n_tiles * blockIdx.x;
    const int2 *Rv = ranges + (int64_t)v * cp.n_tiles;
    const unsigned lt = lanemask_lt();
    uint32_t head = 0, tail = 0;                        // queued: [head, tail), mod EMIT_Q
    // slot counters of a row: the tiles' list starts plus the chunk's offsets
    auto init_row = [&](int row) {
        const uint32_t *h = hc + (int64_t)row * ntx;
        const int2 *R = Rv + (int64_t)row * ntx;
        for (int x = lane; x < NC; x += 32) cnt[x] = x < ntx ? (uint32_t)R[x].x + h[x] : 0u;
        for (int x = lane; x < NC + 4; x += 32) M[x] = 0u;
    };
    // writes the ne (1..32) pairs at the head of the queue
    auto drain = [&](int ne) {
        __syncwarp();
        uint32_t gv = 0u;
        int x0 = 0, w = 0;
        if (lane < ne) {
            const int i = q[(head + lane) % EMIT_Q];
            const uint32_t xs = s_x[i];
            gv = s_g[i];
            x0 = (int)(xs & 0xFFFFu);
            w = (int)(xs >> 16) - x0 + 1;
            atomicXor(&M[x0], 1u << lane);
            atomicXor(&M[x0 + w], 1u << lane);
        }
        head += ne;
        __syncwarp();
        // inclusive XOR prefix along the row: lane l holds columns CPL l ..
        // CPL l + CPL - 1 in registers, one warp scan of the lanes' totals
        uint32_t m[CPL];
#pragma unroll
        for (int k = 0; k < CPL; k += 4) {
            const uint4 t = *reinterpret_cast<const uint4 *>(M + CPL * lane + k);
            m[k] = t.x; m[k + 1] = t.y; m[k + 2] = t.z; m[k + 3] = t.w;
        }
#pragma unroll
        for (int k = 1; k < CPL; ++k) m[k] ^= m[k - 1];
        uint32_t inc = m[CPL - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc ^= t;
        }
        const uint32_t ex = inc ^ m[CPL - 1];
#pragma unroll
        for (int k = 0; k < CPL; k += 4) {
            m[k] ^= ex; m[k + 1] ^= ex; m[k + 2] ^= ex; m[k + 3] ^= ex;
            *reinterpret_cast<uint4 *>(M + CPL * lane + k) = make_uint4(m[k], m[k + 1], m[k + 2], m[k + 3]);
        }
        __syncwarp();
        const int wl = min(w, EMIT_JCAP);
        for (int j = 0; j < wl; ++j) {
            const int x = x0 + j;
            out[cnt[x] + __popc(M[x] & lt)] = gv;
        }
        // columns past EMIT_JCAP: instance I of the concatenated remainders
        // belongs to the pair whose inclusive prefix first exceeds I
        const int rw = max(w - EMIT_JCAP, 0);
        if (__any_sync(0xffffffffu, rw > 0)) {
            int incl = rw;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int base = 0; base < total; base += 32) {
                const int I = base + lane;
                int e = 0;                              // the number of pairs with incl <= I
#pragma unroll
                for (int s = 16; s > 0; s >>= 1) {
                    const int t = __shfl_sync(0xffffffffu, incl, e + s - 1);
                    if (t <= I) e += s;
                }
                const int start = __shfl_sync(0xffffffffu, incl - rw, e);
                const int xe = __shfl_sync(0xffffffffu, x0, e);
                const uint32_t ge = __shfl_sync(0xffffffffu, gv, e);
                if (I < total) {
                    const int x = xe + EMIT_JCAP + (I - start);
                    out[cnt[x] + __popc(M[x] & ((1u << e) - 1u))] = ge;
                }
            }
        }
        __syncwarp();
        // cnt[x] += popc(M[x]) from the registers; M back to zero
#pragma unroll
        for (int k = 0; k < CPL; k += 4) {
            uint4 c = *reinterpret_cast<const uint4 *>(cnt + CPL * lane + k);
            c.x += __popc(m[k]); c.y += __popc(m[k + 1]); c.z += __popc(m[k + 2]); c.w += __popc(m[k + 3]);
            *reinterpret_cast<uint4 *>(cnt + CPL * lane + k) = c;
            *reinterpret_cast<uint4 *>(M + CPL * lane + k) = make_uint4(0u, 0u, 0u, 0u);
        }
        if (lane == 0) M[NC] = 0u;
        __syncwarp();
    };
    // one row over the m staged pairs: 128 pairs per step (four ballots),
    // queued in pair order, written out 32 at a time and emptied at the end
    // (before the stage is replaced; one call site of the drain)
    auto scan_row = [&](int row, int m) {
        const uint32_t rowbit = 1u << (row & 31);
        int i0 = 0;
        while (true) {
            const uint32_t qn = tail - head;            // at most 31 + 128
            if (qn >= 32u || (i0 >= m && qn > 0u)) {
                drain((int)min(qn, 32u));
                continue;
            }
            if (i0 >= m) break;
            bool p[4];
            unsigned b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + 32 * u + lane;
                p[u] = false;
                if (i < m) {
                    const uint32_t y = s_y[i];
                    p[u] = RMASK ? (y & rowbit) != 0u
                                 : (int)(y & 0xFFFFu) <= row && row <= (int)(y >> 16);
                }
                b[u] = __ballot_sync(0xffffffffu, p[u]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (p[u]) q[(tail + __popc(b[u] & lt)) % EMIT_Q] = (uint16_t)(i0 + 32 * u + lane);
                tail += __popc(b[u]);
            }
            i0 += 128;
        }
    };
    const uint32_t *g = sorted_g + L.vd_off[v] + ch.begin;
    const uint2 *sr = srect + L.vd_off[v] + ch.begin;
    auto stage = [&](int s0, int m) {
        for (int j = threadIdx.x; j < m; j += TILE_EMIT_WARPS * 32) {
            const uint2 rc = sr[s0 + j];
            if (RMASK) {
                const uint32_t y0 = rc.y & 0xFFFFu, y1 = rc.y >> 16;     // y0 <= y1 <= 31
                s_y[j] = ((2u << y1) - 1u) & (0xFFFFFFFFu << y0);
            } else {
                s_y[j] = rc.y;
            }
            s_x[j] = rc.x;
            s_g[j] = g[s0 + j];
        }
    };
    if (DYN) {
        const int nty = cp.nty;                         // <= 32; n <= EMIT_STAGE
        if (threadIdx.x < 32) s_load[threadIdx.x] = 0u;
        if (threadIdx.x == 0) s_next = 0;
        stage(0, n);
        __syncthreads();
        // the chunk's instances per row: its tiles' offsets up to the next
        // chunk's (the exclusive prefix over the view's chunks), or up to the
        // tile's total for the view's last chunk
        const bool last = ch.begin + cp.bin_chunk >= ch.nv;
        for (int t = threadIdx.x; t < nty * ntx; t += TILE_EMIT_WARPS * 32) {
            const uint32_t nxt = last ? (uint32_t)(Rv[t].y - Rv[t].x) : hc[(int64_t)cp.n_tiles + t];
            const uint32_t c = nxt - hc[t];
            if (c) atomicAdd(&s_load[t / ntx], c);
        }
        __syncthreads();
        if (warp == 0) {                                // heaviest row first, ties by row
            const uint32_t ld = lane < nty ? s_load[lane] : 0u;
            int rank = 0;
            for (int k = 0; k < nty; ++k) {
                const uint32_t o = __shfl_sync(0xffffffffu, ld, k);
                rank += (o > ld || (o == ld && k < lane)) ? 1 : 0;
            }
            if (lane < nty) s_order[rank] = lane;
        }
        __syncthreads();
        while (true) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&s_next, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k >= nty) break;
            const int row = s_order[k];
            init_row(row);
            scan_row(row, n);
        }
    } else {
        const int row = blockIdx.y * TILE_EMIT_WARPS + warp;
        const bool active = row < cp.nty;
        if (active) init_row(row);
        for (int s0 = 0; s0 < n; s0 += EMIT_STAGE) {
            const int m = min(EMIT_STAGE, n - s0);
            __syncthreads();
            stage(s0, m);
            __syncthreads();
            if (active) scan_row(row, m);
        }
    }
}

__global__ void __launch_bounds__(TILE_EMIT_WARPS * 32)
k_tile_emit_smem(const uint32_t *__restrict__ sorted_g, const uint2 *__restrict__ srect,
                 const uint32_t *__restrict__ n_vis, const uint32_t *__restrict__ n_inst,
                 const uint32_t *__restrict__ bhist, const int2 *__restrict__ ranges, Layout L, CamParams cp,
                 uint32_t *__restrict__ inst_gauss)
{
    __shared__ uint2 s_rc[EMIT_STAGE];
    __shared__ uint32_t s_g[EMIT_STAGE];
    __shared__ uint2 s_q[TILE_EMIT_WARPS][64];
    extern __shared__ uint32_t s_cnt[];                 // [TILE_EMIT_WARPS][ntx]
    const EmitChunk ch = emit_chunk(n_vis, n_inst, L, cp);
    if (ch.skip) return;
    const int v = ch.v, n = ch.n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row = blockIdx.y * TILE_EMIT_WARPS + warp;
    const bool active = row < cp.nty;
    const int ntx = cp.ntx;
    uint2 *q = s_q[warp];
    uint32_t *out = inst_gauss + L.io_off[v];
    uint32_t *cnt = s_cnt + warp * ntx;
    if (active) {
        const uint32_t *h = bhist + (int64_t)cp.n_tiles * blockIdx.x + (int64_t)row * ntx;
        const int2 *R = ranges + (int64_t)v * cp.n_tiles + (int64_t)row * ntx;
        for (int x = lane; x < ntx; x += 32) cnt[x] = (uint32_t)R[x].x + h[x];
    }
    auto drain = [&](int cnt_q) {
        for (int j = 0; j < cnt_q; ++j) {
            const uint2 e = q[j];
            const uint32_t x0 = e.y & 0xFFFFu, x1 = e.y >> 16;
            for (uint32_t x = x0 + (((uint32_t)lane - x0) & 31u); x <= x1; x += 32) {
                const uint32_t p = cnt[x];
                out[p] = e.x;
                cnt[x] = p + 1;
            }
        }
    };
    const uint32_t *g = sorted_g + L.vd_off[v] + ch.begin;
    const uint2 *sr = srect + L.vd_off[v] + ch.begin;
    const unsigned lt = lanemask_lt();
    int qn = 0;
    for (int s0 = 0; s0 < n; s0 += EMIT_STAGE) {
        const int m = min(EMIT_STAGE, n - s0);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += TILE_EMIT_WARPS * 32) {
            s_rc[j] = sr[s0 + j];
            s_g[j] = g[s0 + j];
        }
        __syncthreads();
        if (!active) continue;
        for (int i0 = 0; i0 < m; i0 += 32) {
            const int i = i0 + lane;
            bool p = false;
            uint2 e = make_uint2(0u, 0u);
            if (i < m) {
                const uint2 rc = s_rc[i];
                p = (int)(rc.y & 0xFFFFu) <= row && row <= (int)(rc.y >> 16);
                e = make_uint2(p ? s_g[i] : 0u, rc.x);
            }
            const unsigned mask = __ballot_sync(0xffffffffu, p);
            if (p) q[qn + __popc(mask & lt)] = e;
            qn += __popc(mask);
            if (qn >= 32) {
                __syncwarp();
                drain(qn);
                qn = 0;
                __syncwarp();
            }
        }
    }
    if (active && qn > 0) {
        __syncwarp();
        drain(qn);
    }
}

cudaError_t launch_tile_emit(const uint32_t *sorted_g, const uint2 *srect, const uint32_t *n_vis,
                             const uint32_t *n_inst, const uint32_t *bhist, const int2 *ranges, const Layout &L,
                             const CamParams &cp, int n_chunks, uint32_t *inst_gauss, cudaStream_t st)
{
    if (n_chunks <= 0 || L.V <= 0) return cudaSuccess;
    const dim3 grid(n_chunks, (unsigned)ceil_div(cp.nty, TILE_EMIT_WARPS));
    // a block per chunk needs enough chunks to fill the GPU (a one-view launch
    // has ~80); fewer take a block per (chunk, eight rows)
    const bool rm = cp.nty <= 32, dyn = rm && cp.bin_chunk <= EMIT_STAGE && n_chunks >= EMIT_DYN_MIN_CHUNKS;
    const dim3 grid1(n_chunks, 1);
#define EMIT_FLAT(CPL_)                                                                                         \
    if (dyn)                                                                                                    \
        k_tile_emit_flat<CPL_, true, true><<<grid1, TILE_EMIT_WARPS * 32, 0, st>>>(                             \
            sorted_g, srect, n_vis, n_inst, bhist, ranges, L, cp, inst_gauss);                                  \
    else if (rm)                                                                                                \
        k_tile_emit_flat<CPL_, true, false><<<grid, TILE_EMIT_WARPS * 32, 0, st>>>(                             \
            sorted_g, srect, n_vis, n_inst, bhist, ranges, L, cp, inst_gauss);                                  \
    else                                                                                                        \
        k_tile_emit_flat<CPL_, false, false><<<grid, TILE_EMIT_WARPS * 32, 0, st>>>(                            \
            sorted_g, srect, n_vis, n_inst, bhist, ranges, L, cp, inst_gauss)
    if (cp.ntx <= 128) {
        EMIT_FLAT(4);
    } else if (cp.ntx <= EMIT_FLAT_MAX_NTX) {
        EMIT_FLAT(8);
#undef EMIT_FLAT
    } else {
        const size_t smem = 4 * (size_t)TILE_EMIT_WARPS * cp.ntx;
        k_tile_emit_smem<<<grid, TILE_EMIT_WARPS * 32, smem, st>>>(sorted_g, srect, n_vis, n_inst, bhist, ranges,
                                                                  L, cp, inst_gauss);
    }
    return cudaGetLastError();
}

cudaError_t configure_tile_kernels()
{
    return cudaFuncSetAttribute(k_tile_emit_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_EMIT_SMEM_MAX);
}

// Tile id of every instance of one view, from its ranges (debug export).
__global__ void k_fill_tiles(const int2 *__restrict__ R, int n_tiles, uint32_t *__restrict__ tiles)
{
    const int t = blockIdx.x;
    if (t >= n_tiles) return;
    const int2 r = R[t];
    for (int j = r.x + threadIdx.x; j < r.y; j += blockDim.x) tiles[j] = (uint32_t)t;
}

cudaError_t launch_fill_tiles(const int2 *ranges_view, int n_tiles, uint32_t *tiles_view, cudaStream_t st)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_fill_tiles<<<n_tiles, 128, 0, st>>>(ranges_view, n_tiles, tiles_view);
    return cudaGetLastError();
}

}  // namespace reloc

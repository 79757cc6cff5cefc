// Tile binning and depth sort (GS3LAM Sec. 3.2.1: Gaussians are blended in
// depth order; rasterisation is tile based).
//
// The result is the order of the 64-bit keys (tile << 32 | depth bits) with
// ties broken by item index.  Instead of radix-sorting 64-bit keys over all
// M instances (six 8-bit passes over M), the sort runs in two stages:
//   1. the visible items (tiles_touched > 0) are compacted in index order and
//      sorted by their 32-bit depth bits (four passes over the visible items);
//   2. instances are emitted in that depth order and stably sorted by their
//      tile id (one pass per 8 bits of tile id, two for up to 65536 tiles).
// A stable sort by tile of a depth-ordered, index-tie-broken stream is exactly
// the (tile, depth, index) order.
//
// The digit histograms of every pass are counted by the kernels that write the keys (the
// compaction for the depth keys, the emission for the tile keys) with shared-memory atomics.
// Each radix pass is one kernel: a block ranks its keys (1024 or 2048 in a depth pass, 8192 in a tile
// pass) stably within the block (peer lanes of a digit from match_any + per-warp digit
// counters), publishes its per-digit
// counts, finds its global offsets by a chained look-back over earlier blocks,
// and scatters through shared memory.  Blocks take tile numbers from an atomic
// counter so a block only waits on blocks that are already running; every wait
// is bounded and reports GS_ERR_TIMEOUT in the status word if it gives up.
#include <type_traits>

#include "common.cuh"

namespace gs {

// Counter slots in the workspace.
enum { CTR_NVIS = 0, CTR_M = 1, CTR_MRAW = 2, CTR_TILE = 8 };

namespace {

constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1;

// ----------------------------------------------------------- block scan helper
// Exclusive scan of one value per thread over a block of NT threads (256 unless given);
// returns the prefix and writes the block total to *total.  s_warp holds NT / 32 + 1 values.
template <int NT = 256>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *total, uint32_t *s_warp) {
    constexpr int W = NT / 32;
    static_assert(NT % 32 == 0 && W <= 32, "block of at most 32 warps");
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < W ? s_warp[lane] : 0, ti = t;
#pragma unroll
        for (int o = 1; o < W; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < W) s_warp[lane] = ti - t;
        if (lane == W - 1) s_warp[W] = ti;
    }
    __syncthreads();
    uint32_t r = s_warp[w] + inc - x;
    *total = s_warp[W];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------ state of a call
// Zeroes what a binning accumulates into: the ranges, the counters, the instance count and
// status word, the queued forward's work counters, the tile counts, the emission's per-block
// instance counts, the digit histograms and the look-back flags (the last and largest in 16-byte
// stores over the whole grid).
__global__ void __launch_bounds__(256) bin_init_kernel(uint32_t *ranges, int64_t n_ranges, uint32_t *counters,
                                                       int64_t *n_inst, int32_t *status, uint32_t *tile_counts,
                                                       int64_t n_tiles, uint32_t *emit_sums, int64_t n_emit,
                                                       uint32_t *hist, uint4 *lookback, int64_t n_lookback4,
                                                       uint32_t *queue) {
    pdl_wait();
    pdl_trigger();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = i0; i < n_lookback4; i += stride) lookback[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int64_t i = i0; i < n_ranges; i += stride) ranges[i] = 0u;
    for (int64_t i = i0; i < n_tiles; i += stride) tile_counts[i] = 0u;
    for (int64_t i = i0; i < n_emit; i += stride) emit_sums[i] = 0u;
    for (int64_t i = i0; i < 8 * 256; i += stride) hist[i] = 0u;
    for (int64_t i = i0; i < 64; i += stride) counters[i] = 0u;
    if (i0 == 0) {
        *n_inst = 0;
        *status = 0;
        if (queue) queue[0] = queue[1] = 0u;
    }
}

// ------------------------------------------------ compaction of visible items
__global__ void __launch_bounds__(256) vis_reduce_kernel(const int32_t *touched, int64_t count, uint32_t *block_sums) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ uint32_t s_warp[9];
    int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanIPT;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) c += (base + k < count && touched[base + k] > 0) ? 1u : 0u;
    uint32_t tot;
    block_exclusive_scan(c, &tot, s_warp);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Single-block exclusive scan of nb block sums; total -> counters[slot].
// If cap_slot >= 0 the total is also clamped to capacity into counters[cap_slot],
// the raw count goes to *n_inst and overflow sets the status word.
__global__ void __launch_bounds__(1024) blocksum_scan_kernel(uint32_t *block_sums, const uint32_t *nb_from,
                                                             int64_t nb_fixed, int items_per_block,
                                                             uint32_t *counters, int slot, int cap_slot,
                                                             int64_t capacity, int64_t *n_inst, int32_t *status) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ uint32_t s_part[1024];
    const bool failed = binning_failed(status);
    int64_t nb = nb_from ? ((int64_t)*nb_from + items_per_block - 1) / items_per_block : nb_fixed;
    if (failed) return;  // whole block (the word is only written by earlier kernels)
    int64_t per = (nb + 1023) / 1024;
    int64_t b0 = (int64_t)threadIdx.x * per;
    uint32_t s = 0;
    for (int64_t i = b0; i < b0 + per && i < nb; ++i) s += block_sums[i];
    s_part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        uint32_t y = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0;
        __syncthreads();
        s_part[threadIdx.x] += y;
        __syncthreads();
    }
    uint32_t run = s_part[threadIdx.x] - s;
    for (int64_t i = b0; i < b0 + per && i < nb; ++i) {
        uint32_t x = block_sums[i];
        block_sums[i] = run;
        run += x;
    }
    if (threadIdx.x == 1023) {
        uint32_t total = s_part[1023];
        counters[slot] = total;
        if (cap_slot >= 0) {
            counters[cap_slot] = (int64_t)total > capacity ? (uint32_t)capacity : total;
            if (n_inst) *n_inst = total;
            if ((int64_t)total > capacity) set_status(status, GS_ERR_CAPACITY);
        }
    }
}

// Adds the 8-bit digits of passes [0, n_passes) of `key` (lanes with `valid`) to the block's
// shared histograms.  Every lane of the warp calls it.  Per pass: one atomic for the warp
// when all of its valid lanes have the same digit (the high digits of nearby keys), else one
// per lane (the low digits, mostly distinct, so the atomics rarely collide).
__device__ __forceinline__ void hist_add(uint32_t (*sh)[256], int n_passes, bool valid, uint32_t key) {
    const uint32_t mask = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const int lane = threadIdx.x & 31, first = __ffs(mask) - 1;
    for (int p = 0; p < n_passes; ++p) {
        const uint32_t d = (key >> (8 * p)) & 255u;
        const uint32_t d0 = __shfl_sync(mask, d, first);
        if (__all_sync(mask, d == d0)) {
            if (lane == first) atomicAdd(&sh[p][d], (uint32_t)__popc(mask));
        } else {
            atomicAdd(&sh[p][d], 1u);
        }
    }
}

// Adds the block's shared histograms into the global ones (zero counts skipped).
__device__ __forceinline__ void hist_flush(uint32_t (*sh)[256], int n_passes, uint32_t *hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < n_passes * 256; i += blockDim.x) {
        const uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(&hist[i], c);
    }
}

// Order-preserving compaction of the visible items with their depth keys; also the digit
// histograms of the depth sort's four passes (no separate pass over the keys), counted over the
// block's visible keys gathered in shared memory, so that the warps count only visible keys
// (about a fifth of the items of a frame) in whole rounds of 32.
__global__ void __launch_bounds__(256) vis_compact_kernel(const int32_t *touched, const float4 *uvdo, int64_t count,
                                                          const uint32_t *block_sums, uint32_t *keys, uint32_t *vals,
                                                          uint32_t *hist) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ uint32_t s_warp[9];
    __shared__ uint32_t sh[4][256];
    __shared__ uint32_t s_key[kScanBlock];  // the block's visible keys, in item order
    for (int i = threadIdx.x; i < 4 * 256; i += 256) (&sh[0][0])[i] = 0u;
    int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanIPT;
    bool f[kScanIPT];
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) {
        f[k] = base + k < count && touched[base + k] > 0;
        c += f[k];
    }
    uint32_t tot;
    uint32_t loc = block_exclusive_scan(c, &tot, s_warp);
    uint32_t off = block_sums[blockIdx.x] + loc;
#pragma unroll
    for (int k = 0; k < kScanIPT; ++k) {
        if (f[k]) {
            const uint32_t key = __float_as_uint(uvdo[base + k].z);
            keys[off] = key;
            vals[off] = (uint32_t)(base + k);
            s_key[loc] = key;
            ++off;
            ++loc;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (uint32_t i0 = threadIdx.x - lane; i0 < tot; i0 += 256) {  // warp-uniform rounds
        const uint32_t i = i0 + lane;
        hist_add(sh, 4, i < tot, i < tot ? s_key[i] : 0u);
    }
    hist_flush(sh, 4, hist);
}

// ------------------------------------------------------------ instance emission
constexpr int kEmitBlock = 256;  // sorted items per block of the emission kernels

// One thread per sorted item computes its instance offset; the block's instances are then
// split evenly over its warps, 32 consecutive instances per warp round, each lane finding
// the item that owns its instance by a binary search over the block's item offsets in
// shared memory.  Every store is coalesced, and a few long items (large splats) no longer
// keep one warp of the block busy while the others idle.
// Also the digit histograms of the tile sort's n_passes passes over the written keys.
__global__ void __launch_bounds__(kEmitBlock) emit_kernel(ViewTable vt, const uint32_t *sorted_items,
                                                          const int32_t *touched, const float4 *uvdo,
                                                          const float4 *conic, const uint32_t *counters,
                                                          const uint32_t *block_sums, int64_t capacity,
                                                          uint32_t *tile_keys, uint32_t *inst_vals, int n_passes,
                                                          uint32_t *hist, int64_t vn, const int32_t *status) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ uint32_t s_warp[9];
    __shared__ uint32_t sh[4][256];
    __shared__ uint32_t s_off[kEmitBlock];   // exclusive instance offset of each item in the block
    __shared__ uint32_t s_item[kEmitBlock];
    __shared__ uint4 s_rect[kEmitBlock];     // (x0, y0, width, tiles per row | first tile of the view << 16)
    // whole block (the word is only written by earlier kernels): after a failed depth sort or an
    // overflow nothing is emitted
    const bool failed = binning_failed(status);
    const int64_t count = counters[CTR_NVIS];
    if (failed || (int64_t)blockIdx.x * kEmitBlock >= count) return;  // whole block: no barrier is skipped
    for (int i = threadIdx.x; i < 4 * 256; i += kEmitBlock) (&sh[0][0])[i] = 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kEmitBlock + threadIdx.x;
    uint32_t item = 0, c = 0;
    int x0 = 0, y0 = 0, w = 1, tx = 1;
    uint32_t tb = 0;
    if (i < count && sorted_items[i] < vn) {
        item = sorted_items[i];
        c = (uint32_t)touched[item];
        const int v = (int)(item / (uint32_t)vt.n);
        const float4 rec = uvdo[item];
        int x1, y1;
        tile_rect(rec.x, rec.y, (int)conic[item].w, vt.TX[v], vt.TY[v], x0, y0, x1, y1);
        w = max(x1 - x0, 1);
        tx = vt.TX[v];
        tb = (uint32_t)vt.tile_off[v];
    }
    uint32_t tot;
    const uint32_t excl = block_exclusive_scan(c, &tot, s_warp);
    s_off[threadIdx.x] = excl;
    s_item[threadIdx.x] = item;
    s_rect[threadIdx.x] = make_uint4((uint32_t)x0, (uint32_t)y0, (uint32_t)w, (uint32_t)tx);
    if (threadIdx.x == 0) s_warp[8] = tot;
    __shared__ uint32_t s_tb[kEmitBlock];
    s_tb[threadIdx.x] = tb;
    __syncthreads();
    const uint32_t bbase = block_sums[blockIdx.x];
    // warp wid takes instances [q_lo, q_hi) of the block, in whole rounds of 32
    const uint32_t per = ((tot + 32u * (kEmitBlock / 32) - 1) / (32u * (kEmitBlock / 32))) * 32u;
    const uint32_t q_lo = min(tot, (uint32_t)wid * per), q_hi = min(tot, q_lo + per);
    for (uint32_t q0 = q_lo; q0 < q_hi; q0 += 32) {
        const uint32_t q = q0 + lane;
        const bool valid = q < q_hi;
        // the owner: the last item whose offset is <= q (items with no instances share offsets)
        int owner = 0;
#pragma unroll
        for (int step = kEmitBlock / 2; step >= 1; step >>= 1)
            if (s_off[owner + step] <= q) owner += step;
        const int64_t off = (int64_t)bbase + q;
        const bool write = valid && off < capacity;
        uint32_t key = 0u;
        if (write) {
            const uint4 rc = s_rect[owner];
            const int k = (int)(q - s_off[owner]);
            const int ky = k / (int)rc.z, kx = k - ky * (int)rc.z;
            key = s_tb[owner] + (uint32_t)(((int)rc.y + ky) * (int)rc.w + (int)rc.x + kx);
            tile_keys[off] = key;
            inst_vals[off] = s_item[owner];
        }
        hist_add(sh, n_passes, write, key);
    }
    hist_flush(sh, n_passes, hist);
}

// ------------------------------------------------------------------ radix sort
// Shared memory of a radix-pass block of NT threads with IPT keys each (dynamic: 99 KB for 1024 x 8).
template <int NT, int IPT>
struct SortSmem {
    uint32_t keys[NT * IPT];
    uint32_t vals[NT * IPT];
    uint32_t whist[NT / 32][256];
    uint32_t excl[256];   // block-local exclusive digit offsets
    uint32_t glob[256];   // global destination of the digit's first key in this block
    uint32_t dbase[256];  // global exclusive digit base of the pass
    uint32_t warp[NT / 32 + 1];
    uint32_t tile;
    int failed;
};

// One radix pass, NT threads per block and IPT keys per thread: 256 threads for the depth
// passes over the visible items, 1024 for the tile passes over the instances, where a quarter
// as many blocks means a sixteenth of the look-back's reads (every block starts at once and
// reads back through about half of the blocks before it).
// Resident blocks per SM the register allocation must allow: four depth-pass blocks of 8 keys a
// thread (64 registers), six of 4 (40); two tile-pass blocks (32 registers, about 100 bytes
// spilled, which costs less than a second wave of blocks: tile sort 0.179 -> 0.172 ms on 2.2 M
// instances).
template <int NT, int IPT> constexpr int sort_min_blocks() {
    return NT == 256 ? (IPT >= 8 ? 4 : 6) : (NT == 512 ? 3 : 2);
}

template <int NT, int IPT>
__global__ void __launch_bounds__(NT, sort_min_blocks<NT, IPT>()) onesweep_kernel(const uint32_t *keys_in, const uint32_t *vals_in,
                                                      uint32_t *keys_out, uint32_t *vals_out,
                                                      const uint32_t *count_ptr, int shift,
                                                      const uint32_t *pass_hist, uint32_t *tile_ctr,
                                                      uint32_t *lookback, int32_t *status, int spin_limit,
                                                      uint32_t *tile_counts, uint32_t n_tiles,
                                                      const int32_t *emit_touched, uint32_t *emit_sums,
                                                      uint32_t emit_vn) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    constexpr int W = NT / 32, TILE = NT * IPT;
    static_assert(NT >= 256, "one thread per digit");
    extern __shared__ __align__(16) unsigned char sort_smem[];
    SortSmem<NT, IPT> &S = *reinterpret_cast<SortSmem<NT, IPT> *>(sort_smem);
    uint32_t *s_keys = S.keys, *s_vals = S.vals, *s_excl = S.excl, *s_glob = S.glob, *s_dbase = S.dbase;
    uint32_t(*s_whist)[256] = S.whist;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        S.tile = atomicAdd(tile_ctr, 1u);
        S.failed = binning_failed(status);
    }
    for (int i = tid; i < W * 256; i += NT) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = S.tile;
    if (S.failed) {
        // an earlier wait gave up (or the count overflowed): this pass's output is not used.  The
        // block still publishes an inclusive prefix (0: never more than the true one, so a block
        // that adds it scatters in bounds) so that no running block waits for it.
        if (tid < 256) st_relaxed(lookback + (size_t)tile * 256 + tid, kFlagPre);
        return;
    }
    const int64_t n = *count_ptr;
    const int64_t base = (int64_t)tile * TILE;
    if (base >= n) return;

    uint32_t key[IPT], val[IPT], rank[IPT];
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
        const int64_t i = base + (int64_t)w * (IPT * 32) + r * 32 + lane;
        key[r] = i < n ? keys_in[i] : 0u;
        val[r] = i < n ? vals_in[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
        const bool valid = base + (int64_t)w * (IPT * 32) + r * 32 + lane < n;
        const uint32_t d = (key[r] >> shift) & 255u;
        // lanes with the same digit; an invalid lane matches only itself
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 256u + lane);
        int leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if (valid && lane == leader) {
            b = s_whist[w][d];
            s_whist[w][d] = b + __popc(peers);
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        rank[r] = b + __popc(peers & lanemask_lt());
        __syncwarp();
    }
    __syncthreads();

    // per-digit (thread d < 256): warp-exclusive offsets and the block's count, published at once
    // for later tiles
    const int d = tid;
    uint32_t cnt = 0, hist_d = 0;
    uint32_t *my = lookback + (size_t)tile * 256 + (d & 255);
    if (d < 256) {
#pragma unroll
        for (int ww = 0; ww < W; ++ww) {
            uint32_t c = s_whist[ww][d];
            s_whist[ww][d] = cnt;
            cnt += c;
        }
        st_relaxed(my, (tile == 0 ? kFlagPre : kFlagAgg) | cnt);
        hist_d = pass_hist[d];
    }
    // block-exclusive digit offsets and the pass's digit bases
    uint32_t lb_tot;
    const uint32_t ex = block_exclusive_scan<NT>(cnt, &lb_tot, S.warp);
    if (d < 256) s_excl[d] = ex;
    uint32_t hist_tot;
    const uint32_t db = block_exclusive_scan<NT>(hist_d, &hist_tot, S.warp);  // its barriers publish s_excl
    if (d < 256) s_dbase[d] = db;

    // local scatter by digit into shared memory (the keys leave the registers before the wait)
#pragma unroll
    for (int r = 0; r < IPT; ++r) {
        int64_t i = base + (int64_t)w * (IPT * 32) + r * 32 + lane;
        if (i < n) {
            uint32_t dd = (key[r] >> shift) & 255u;
            uint32_t pos = s_excl[dd] + s_whist[w][dd] + rank[r];
            s_keys[pos] = key[r];
            s_vals[pos] = val[r];
        }
    }

    // chained look-back over earlier tiles for digit d: kWin of their flags are read at a time
    // (all tiles start together, so the chain is as long as the tile number over kWin); spin
    // (bounded) only on a tile that has not published its count yet
    uint32_t prefix = 0;
    if (tile != 0 && d < 256) {
        constexpr int kWin = 8;
        int64_t t = (int64_t)tile - 1;
        bool done = false, timeout = false;
        while (!done && t >= 0) {
            uint32_t w[kWin];
#pragma unroll
            for (int i = 0; i < kWin; ++i) w[i] = t - i >= 0 ? ld_relaxed(lookback + (size_t)(t - i) * 256 + d) : 0u;
#pragma unroll
            for (int i = 0; i < kWin; ++i) {
                if (done) continue;
                if (t - i < 0 || spin_limit < 0) {  // the first tile passed; or the test hook: give up at once
                    timeout = spin_limit < 0;
                    done = true;
                    continue;
                }
                uint32_t vv = w[i];
                if ((vv & ~kValMask) == 0u) {
                    const uint32_t *pp = lookback + (size_t)(t - i) * 256 + d;
                    int spin = 0;
                    while ((vv & ~kValMask) == 0u && spin < spin_limit) {
                        if (++spin > 64) __nanosleep(64);
                        vv = ld_relaxed(pp);
                    }
                    if ((vv & ~kValMask) == 0u) {
                        timeout = true;
                        done = true;
                        continue;
                    }
                }
                prefix += vv & kValMask;
                if ((vv & ~kValMask) == kFlagPre) done = true;
            }
            t -= kWin;
        }
        if (timeout) set_status(status, GS_ERR_TIMEOUT);
        st_relaxed(my, kFlagPre | (prefix + cnt));
    }
    if (d < 256) s_glob[d] = s_dbase[d] + prefix;
    __syncthreads();

    // coalesced-by-run global writes, in warp-uniform rounds of 32 consecutive keys
    const int tile_n = (int)min((int64_t)TILE, n - base);
    for (int i0 = tid - lane; i0 < tile_n; i0 += NT) {
        const int i = i0 + lane;
        const bool ok = i < tile_n;
        uint32_t dst = 0u, v = 0u;
        if (ok) {
            const uint32_t k = s_keys[i];
            const uint32_t dd = (k >> shift) & 255u;
            dst = s_glob[dd] + (uint32_t)i - s_excl[dd];
            v = s_vals[i];
            keys_out[dst] = k;
            vals_out[dst] = v;
            // last pass of the tile sort: the block's keys are sorted by tile here, so each run of one
            // tile adds its length to the tile's count (end + 1 from its last key, -start from its first)
            if (tile_counts && k < n_tiles) {
                if (i == 0 || s_keys[i - 1] != k) atomicAdd(&tile_counts[k], 0u - (uint32_t)i);
                if (i == tile_n - 1 || s_keys[i + 1] != k) atomicAdd(&tile_counts[k], (uint32_t)i + 1u);
            }
        }
        if (emit_sums) {
            // last pass of the depth sort: the instances of each block of kEmitBlock sorted items,
            // which the emission scans.  dst increases with i in a block (digits in order, each
            // digit's keys at consecutive places), so the lanes of one emission block are
            // consecutive: a segmented sum over the warp and one atomic per segment.
            const uint32_t seg = ok ? dst / (uint32_t)kEmitBlock : 0xffffffffu;
            uint32_t c = ok && v < emit_vn ? (uint32_t)emit_touched[v] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, c, o);
                const uint32_t sy = __shfl_up_sync(0xffffffffu, seg, o);
                if (lane >= o && sy == seg) c += y;
            }
            const uint32_t s_next = __shfl_down_sync(0xffffffffu, seg, 1);
            if (ok && (lane == 31 || s_next != seg) && c) atomicAdd(&emit_sums[seg], c);
        }
    }
}

// The optional 64-bit keys (tile << 32 | depth bits) of the sorted instances.  Tile ids and
// items are checked against their counts: only a sort that gave up (status set, so nothing
// runs here) could leave other values, but an access out of bounds must not be possible.
__global__ void __launch_bounds__(256) keys64_kernel(const uint32_t *tile_keys, const uint32_t *vals,
                                                     const uint32_t *counters, const float4 *uvdo, uint64_t *keys64,
                                                     int64_t n_tiles, int64_t vn, const int32_t *status) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    const bool failed = binning_failed(status);
    int64_t m = counters[CTR_M];
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (failed || j >= m) return;
    const uint32_t t = tile_keys[j], it = vals[j];
    keys64[j] = t < n_tiles && it < vn ? ((uint64_t)t << 32) | __float_as_uint(uvdo[it].z) : ~0ull;
}

struct SortBufs {
    uint32_t *k0, *v0, *k1, *v1;
};

// Stable LSD sort of (key, val) pairs by `n_passes` 8-bit digits from bit 0, given the
// digit histograms of every pass (hist [n_passes][256], written by the kernel that
// produced the keys).  Input in (k0, v0); output lands in (k0, v0) if n_passes is even,
// else (k1, v1).  The last pass also adds the tile runs to tile_counts and, with emit_sums,
// emit_touched[val] to the count of its kEmitBlock-item block of the output (either optional).
template <int NT, int IPT>
gs_status radix_sort(SortBufs b, const uint32_t *count_ptr, int64_t max_count, int n_passes, const uint32_t *hist,
                     uint32_t *lookback, int lb_tiles, uint32_t *tile_ctrs, int32_t *status, int spin_limit,
                     cudaStream_t st, uint32_t *tile_counts = nullptr, uint32_t n_tiles = 0,
                     const int32_t *emit_touched = nullptr, uint32_t *emit_sums = nullptr, uint32_t emit_vn = 0) {
    if (max_count <= 0 || n_passes <= 0) return GS_OK;
    constexpr size_t smem = sizeof(SortSmem<NT, IPT>);
    if (smem > 48 * 1024) {
        // above the static limit: opted in once per device
        static bool opted[64] = {false};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return GS_ERR_CUDA;
        if (dev < 0 || dev >= 64 || !opted[dev]) {
            if (cudaFuncSetAttribute(onesweep_kernel<NT, IPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess)
                return GS_ERR_CUDA;
            if (dev >= 0 && dev < 64) opted[dev] = true;
        }
    }
    int grid = ceil_div(max_count, (int64_t)NT * IPT);
    uint32_t *ki = b.k0, *vi = b.v0, *ko = b.k1, *vo = b.v1;
    for (int p = 0; p < n_passes; ++p) {
        const gs_status s = launch_pdl(onesweep_kernel<NT, IPT>, grid, NT, smem, st, ki, vi, ko, vo, count_ptr, 8 * p,
                                       hist + 256 * p, tile_ctrs + p, lookback + (size_t)p * lb_tiles * 256, status,
                                       spin_limit, p == n_passes - 1 ? tile_counts : nullptr, n_tiles, emit_touched,
                                       p == n_passes - 1 ? emit_sums : nullptr, emit_vn);
        if (s) return s;
        uint32_t *tk = ki, *tv = vi;
        ki = ko; vi = vo; ko = tk; vo = tv;
    }
    return last_launch();
}

}  // namespace
}  // namespace gs

namespace gs {
namespace {

// Per-tile ranges and the launch order of the blend kernels' tiles, from the instance count of
// every tile (counted by the last tile-sort pass).  One CTA of 1024 threads.
//   ranges: an exclusive scan of the counts (each thread scans a contiguous chunk of tiles),
//   [0, 0) for an empty tile;
//   order: decreasing instance count, so the longest tiles start first and the short ones fill
//   in behind them (longest-processing-time-first; the order within a count bucket is
//   arbitrary): a counting sort on a bucket of the count (exact below 1024 instances,
//   64-instance steps above, saturating at 50,112), buckets taken high to low.
// After a failed binning the ranges stay empty and every count is taken as 0.
__device__ __forceinline__ int order_bucket(uint32_t c) {
    return c < 1024u ? (int)(c >> 2) : (int)min(256u + ((c - 1024u) >> 6), 1023u);
}

// Exclusive scan of one value per thread over the 1024-thread block; returns the prefix.
__device__ __forceinline__ uint32_t scan1024(uint32_t x, uint32_t *warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t t = warp_tot[lane];
        uint32_t ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, ti, d);
            if (lane >= d) ti += y;
        }
        warp_tot[lane] = ti - t;  // exclusive over warps
    }
    __syncthreads();
    const uint32_t r = warp_tot[wid] + inc - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) ranges_order_kernel(const uint32_t *counts, int n_tiles, uint32_t *ranges,
                                                            uint32_t *order, const int32_t *status) {
    pdl_wait();     // the previous kernel's results
    pdl_trigger();  // the next kernel may be scheduled now
    __shared__ uint32_t hist[1024];
    __shared__ uint32_t warp_tot[32];
    const int tid = threadIdx.x;
    const bool failed = binning_failed(status);
    const int per = (n_tiles + 1023) / 1024, t0 = tid * per, t1 = min(n_tiles, t0 + per);
    uint32_t sum = 0;
    for (int t = t0; t < t1; ++t) sum += failed ? 0u : counts[t];
    uint32_t run = scan1024(sum, warp_tot);
    if (!failed)
        for (int t = t0; t < t1; ++t) {
            const uint32_t c = counts[t];
            ranges[2 * t] = c ? run : 0u;  // empty tiles: [0, 0)
            ranges[2 * t + 1] = c ? run + c : 0u;
            run += c;
        }
    if (!order) return;  // whole block
    hist[tid] = 0u;
    __syncthreads();
    for (int t = tid; t < n_tiles; t += 1024) atomicAdd(&hist[order_bucket(failed ? 0u : counts[t])], 1u);
    __syncthreads();
    // exclusive scan over buckets from the highest down: thread i takes bucket 1023 - i
    const uint32_t h = hist[1023 - tid];
    const uint32_t before = scan1024(h, warp_tot);
    hist[1023 - tid] = before;  // first slot of bucket 1023 - tid
    __syncthreads();
    for (int t = tid; t < n_tiles; t += 1024) {
        const uint32_t pos = atomicAdd(&hist[order_bucket(failed ? 0u : counts[t])], 1u);
        order[pos] = (uint32_t)t;
    }
}

gs_status write_ranges_order(const uint32_t *counts, const gs_binning *out, int64_t total_tiles, cudaStream_t st) {
    return launch_pdl(ranges_order_kernel, 1, 1024, 0, st, counts, (int)total_tiles, out->ranges, out->tile_order,
                      out->status);
}

}  // namespace
}  // namespace gs

extern "C" gs_status gs_bin_sort(int64_t n, const gs_projected *proj, const gs_camera *cams, int n_views,
                                 const gs_raster_params *p, void *ws, size_t ws_bytes, gs_binning *out,
                                 gs_stream stream) {
    GS_NVTX_RANGE("gs_bin_sort");
    using namespace gs;
    cudaStream_t st = (cudaStream_t)stream;
    ViewTable vt;
    Params prm;
    if (!proj || !out || n < 0) return GS_ERR_ARG;
    if (!make_view_table(cams, n_views, n, &vt) || !make_params(p, &prm)) return GS_ERR_ARG;
    if (out->capacity < 0 || out->capacity >= ((int64_t)1 << 30) || n * n_views >= ((int64_t)1 << 30)) return GS_ERR_ARG;
    if (!out->vals || !out->ranges || !out->n_inst || !out->status || !ws) return GS_ERR_ARG;
    WsLayout L = ws_layout(n, n_views, out->capacity, &vt);
    if (ws_bytes < L.bin_end || (reinterpret_cast<uintptr_t>(ws) & 255)) return GS_ERR_ARG;
    char *w = static_cast<char *>(ws);
    uint32_t *counters = reinterpret_cast<uint32_t *>(w + L.counters);
    uint32_t *block_sums = reinterpret_cast<uint32_t *>(w + L.scan_blocks);
    uint32_t *emit_sums = reinterpret_cast<uint32_t *>(w + L.emit_sums);
    uint32_t *hist = reinterpret_cast<uint32_t *>(w + L.hist);
    uint32_t *lookback = reinterpret_cast<uint32_t *>(w + L.lookback);
    uint32_t *tile_counts = reinterpret_cast<uint32_t *>(w + L.tile_counts);
    int64_t total_tiles = vt.tile_off[n_views];
    int64_t vn = n * n_views;

    if (vn > 0 && (!proj->uvdo || !proj->conic || !proj->tiles_touched)) return GS_ERR_ARG;

    // Every kernel of the binning is launched with programmatic stream serialization: it is
    // scheduled while its predecessor drains and waits for it (pdl_wait) before reading.
    gs_status s;
    const int64_t n_lb4 = vn > 0 ? 64 * ((int64_t)4 * L.lb_tiles_depth + (int64_t)3 * L.lb_tiles_inst) : 0;
    const int init_grid = (int)std::max<int64_t>(1, std::min<int64_t>((n_lb4 + 255) / 256, 1216));
    const int64_t nbe = ceil_div(vn, kEmitBlock);  // emission blocks
    if ((s = launch_pdl(bin_init_kernel, init_grid, 256, 0, st, out->ranges, 2 * total_tiles, counters, out->n_inst,
                        out->status, tile_counts, total_tiles, emit_sums, nbe + 1, hist,
                        reinterpret_cast<uint4 *>(lookback), n_lb4, out->queue)))
        return s;
    if (vn == 0) return write_ranges_order(tile_counts, out, total_tiles, st);

    const float4 *uvdo = reinterpret_cast<const float4 *>(proj->uvdo);
    const float4 *conic = reinterpret_cast<const float4 *>(proj->conic);
    uint32_t *dk_a = reinterpret_cast<uint32_t *>(w + L.dkeys_a), *dv_a = reinterpret_cast<uint32_t *>(w + L.dvals_a);
    uint32_t *dk_b = reinterpret_cast<uint32_t *>(w + L.dkeys_b), *dv_b = reinterpret_cast<uint32_t *>(w + L.dvals_b);

    // 1. compact visible items in index order, keyed by depth bits
    int nb = ceil_div(vn, kScanBlock);
    if ((s = launch_pdl(vis_reduce_kernel, nb, 256, 0, st, proj->tiles_touched, vn, block_sums))) return s;
    if ((s = launch_pdl(blocksum_scan_kernel, 1, 1024, 0, st, block_sums, nullptr, (int64_t)nb, kScanBlock, counters,
                        (int)CTR_NVIS, -1, (int64_t)0, nullptr, nullptr)))
        return s;
    if ((s = launch_pdl(vis_compact_kernel, nb, 256, 0, st, proj->tiles_touched, uvdo, vn, block_sums, dk_a, dv_a,
                        hist)))
        return s;

    // 2. stable sort of the visible items by depth (4 passes: result in dk_a/dv_a); the last pass
    //    also counts the instances of every emission block of the sorted items
    auto depth_sort = [&](auto ipt) {
        return radix_sort<kSortThreads, decltype(ipt)::value>(
            {dk_a, dv_a, dk_b, dv_b}, counters + CTR_NVIS, vn, 4, hist, lookback, L.lb_tiles_depth, counters + CTR_TILE,
            out->status, prm.spin_limit, st, nullptr, 0, proj->tiles_touched, emit_sums, (uint32_t)vn);
    };
    s = vn <= kSortSmallItems ? depth_sort(std::integral_constant<int, kSortIPTSmall>())
                              : depth_sort(std::integral_constant<int, kSortIPTLarge>());
    if (s) return s;
    const uint32_t *sorted_items = dv_a;

    // 3. emit instances in depth order; instance count -> n_inst (clamped copy for the sort)
    int tile_bits = 1;
    while (((int64_t)1 << tile_bits) < total_tiles) ++tile_bits;
    int tile_passes = (tile_bits + 7) / 8;
    uint32_t *tk_a = reinterpret_cast<uint32_t *>(w + L.tkeys_a), *tk_b = reinterpret_cast<uint32_t *>(w + L.tkeys_b);
    uint32_t *tv_b = reinterpret_cast<uint32_t *>(w + L.tvals_b);
    // the emitted values go where the final pass must not land: out->vals ends the sort
    uint32_t *emit_vals = (tile_passes % 2 == 0) ? out->vals : tv_b;
    uint32_t *other_vals = (tile_passes % 2 == 0) ? tv_b : out->vals;
    if ((s = launch_pdl(blocksum_scan_kernel, 1, 1024, 0, st, emit_sums, counters + CTR_NVIS, (int64_t)0, kEmitBlock,
                        counters, (int)CTR_MRAW, (int)CTR_M, out->capacity, out->n_inst, out->status)))
        return s;
    if ((s = launch_pdl(emit_kernel, (int)nbe, kEmitBlock, 0, st, vt, sorted_items, proj->tiles_touched, uvdo, conic,
                        counters, emit_sums, out->capacity, tk_a, emit_vals, tile_passes, hist + 4 * 256, vn,
                        out->status)))
        return s;
    if (out->capacity == 0) return write_ranges_order(tile_counts, out, total_tiles, st);

    // 4. stable sort of the instances by tile id
    if ((s = radix_sort<kSortThreadsInst, kSortIPTInst>({tk_a, emit_vals, tk_b, other_vals}, counters + CTR_M, out->capacity, tile_passes,
                        hist + 4 * 256, lookback + (size_t)4 * L.lb_tiles_depth * 256, L.lb_tiles_inst,
                        counters + CTR_TILE + 4, out->status, prm.spin_limit, st, tile_counts, (uint32_t)total_tiles)))
        return s;
    const uint32_t *sorted_tiles = (tile_passes % 2 == 0) ? tk_a : tk_b;

    // 5. per-tile ranges from the tile counts, the launch order, and the 64-bit keys if requested
    if ((s = write_ranges_order(tile_counts, out, total_tiles, st))) return s;
    if (out->keys) {
        if ((s = launch_pdl(keys64_kernel, ceil_div(out->capacity, 256), 256, 0, st, sorted_tiles, out->vals, counters,
                            uvdo, out->keys, total_tiles, vn, out->status)))
            return s;
    }
    return GS_OK;
}

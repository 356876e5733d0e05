// bh_sort.cu -- root cube, Morton keys and the onesweep radix sort.
//
// Sec. 4.1: the root cell is a cube enclosing every particle (origin = the
// per-axis minimum, side = the largest extent).  Sec. 5: particles are put in
// Morton order, here by a stable least-significant-digit radix sort of 30-bit
// keys in the single-pass "onesweep" form (Adinets & Merrill 2022): one
// upfront histogram pass fused into key generation, then one kernel per 8-bit
// digit that ranks a tile, resolves its global offsets by decoupled look-back
// and scatters through shared memory.  The last pass also gathers the float4
// particles into Morton order.
#include "bh_internal.cuh"

namespace bh {

// ------------------------------------------------------------ init / bbox

__global__ void bh_init_kernel(bh_dev_ctrl* c)
{
    const int t = threadIdx.x;
    if (t < 3) {
        c->minmax[t] = 0xffffffffu;
        c->minmax[3 + t] = 0u;
    }
    for (int i = t; i < 8 * 256; i += blockDim.x) (&c->hist[0][0])[i] = 0u;
    if (t < 8) c->tile_ctr[t] = 0u;
    if (t == 0) c->scan_done = 0u;
    if (t < BH_LEVEL_SLOTS) {
        c->level_total[t] = 0u;
        c->level_offset[t] = 0u;
    }
    if (t == 0) {
        c->n_nodes = 0u;
        c->status = 0u;
        c->abort = 0u;
        c->n_leaves = 0u;
        c->max_leaf = 0u;
        c->n_groups = 0u;
        c->group_ctr = 0u;
        c->n_pp = 0ull;
        c->n_pc = 0ull;
        c->build_seq += 1u;  // new look-back epochs for this build's sort passes
    }
}

void launch_init(bh_dev_ctrl* ctrl, cudaStream_t s) { bh_init_kernel<<<1, 256, 0, s>>>(ctrl); }

// Per-axis min/max over all particles; flags NaN/Inf coordinates or masses.
__global__ void __launch_bounds__(256) bh_bbox_kernel(const float4* __restrict__ pos, int n, bh_dev_ctrl* c)
{
    unsigned int lo0 = 0xffffffffu, lo1 = 0xffffffffu, lo2 = 0xffffffffu, hi0 = 0u, hi1 = 0u, hi2 = 0u;
    bool bad = false;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w));
        const unsigned int ox = bh_f2ord(p.x), oy = bh_f2ord(p.y), oz = bh_f2ord(p.z);
        lo0 = min(lo0, ox); lo1 = min(lo1, oy); lo2 = min(lo2, oz);
        hi0 = max(hi0, ox); hi1 = max(hi1, oy); hi2 = max(hi2, oz);
    }
    // warp, then block reduction: one set of atomics per block (the six
    // words are shared by every block, so per-warp atomics contended in L2)
    __shared__ unsigned int red[8][7];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    lo0 = __reduce_min_sync(BH_FULL_MASK, lo0);
    lo1 = __reduce_min_sync(BH_FULL_MASK, lo1);
    lo2 = __reduce_min_sync(BH_FULL_MASK, lo2);
    hi0 = __reduce_max_sync(BH_FULL_MASK, hi0);
    hi1 = __reduce_max_sync(BH_FULL_MASK, hi1);
    hi2 = __reduce_max_sync(BH_FULL_MASK, hi2);
    const unsigned int anybad = __any_sync(BH_FULL_MASK, bad) ? 1u : 0u;
    if (lane == 0) {
        red[w][0] = lo0; red[w][1] = lo1; red[w][2] = lo2;
        red[w][3] = hi0; red[w][4] = hi1; red[w][5] = hi2;
        red[w][6] = anybad;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        const bool ok = lane < nw;
        lo0 = __reduce_min_sync(BH_FULL_MASK, ok ? red[lane][0] : 0xffffffffu);
        lo1 = __reduce_min_sync(BH_FULL_MASK, ok ? red[lane][1] : 0xffffffffu);
        lo2 = __reduce_min_sync(BH_FULL_MASK, ok ? red[lane][2] : 0xffffffffu);
        hi0 = __reduce_max_sync(BH_FULL_MASK, ok ? red[lane][3] : 0u);
        hi1 = __reduce_max_sync(BH_FULL_MASK, ok ? red[lane][4] : 0u);
        hi2 = __reduce_max_sync(BH_FULL_MASK, ok ? red[lane][5] : 0u);
        const unsigned int nb = __reduce_or_sync(BH_FULL_MASK, ok ? red[lane][6] : 0u);
        if (lane == 0) {
            atomicMin(&c->minmax[0], lo0);
            atomicMin(&c->minmax[1], lo1);
            atomicMin(&c->minmax[2], lo2);
            atomicMax(&c->minmax[3], hi0);
            atomicMax(&c->minmax[4], hi1);
            atomicMax(&c->minmax[5], hi2);
            if (nb) atomicCAS(&c->status, 0u, (unsigned int)(-BH_ERR_NONFINITE));
        }
    }
}

void launch_bbox(const float4* pos, int n, bh_dev_ctrl* ctrl, int grid, cudaStream_t s)
{
    bh_bbox_kernel<<<grid, 256, 0, s>>>(pos, n, ctrl);
}

// ------------------------------------------------------------------ keys
// q = (x - xmin) * (1024 / L) as two separately rounded FP32 operations,
// c = min(trunc(q), 1023); bit k of cx, cy, cz -> key bit 3k+2, 3k+1, 3k.
// The four digit histograms of the sort (bits 0-7, 8-15, 16-23, 24-29) are
// accumulated on the way.
template <int CURVE, typename K>
__global__ void __launch_bounds__(256) bh_keys_kernel(const float4* __restrict__ pos, int n, bh_dev_ctrl* c,
                                                      K* __restrict__ keys)
{
    constexpr int B = bh_key_traits<K>::kMaxLevel, NP = bh_key_traits<K>::kPasses;
    constexpr unsigned int CMAX = (1u << B) - 1u;
    __shared__ unsigned int sh[NP][256];
    __shared__ float sbox[4];
    __shared__ float sinv;
    for (int i = threadIdx.x; i < NP * 256; i += blockDim.x) (&sh[0][0])[i] = 0u;
    if (threadIdx.x == 0) {
        bh_box_from_minmax(c->minmax, sbox, &sinv);
        if (blockIdx.x == 0) {
            c->box[0] = sbox[0];
            c->box[1] = sbox[1];
            c->box[2] = sbox[2];
            c->box[3] = sbox[3];
            c->inv = sinv;
        }
    }
    __syncthreads();
    // 2^(B - 10) * (1024 / L): the power of two is exact, so the 10-bit cell is the B-bit cell >> (B - 10)
    const float x0 = sbox[0], y0 = sbox[1], z0 = sbox[2], inv = __fmul_rn(sinv, (float)(1u << (B - 10)));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = pos[i];
        const unsigned int cx = min(__float2uint_rz(__fmul_rn(__fsub_rn(p.x, x0), inv)), CMAX);
        const unsigned int cy = min(__float2uint_rz(__fmul_rn(__fsub_rn(p.y, y0), inv)), CMAX);
        const unsigned int cz = min(__float2uint_rz(__fmul_rn(__fsub_rn(p.z, z0), inv)), CMAX);
        const K k = bh_key_of<CURVE, K>(cx, cy, cz);
        keys[i] = k;
#pragma unroll
        for (int d = 0; d < NP; d++) atomicAdd(&sh[d][(unsigned int)(k >> (8 * d)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NP * 256; i += blockDim.x) {
        const unsigned int v = (&sh[0][0])[i];
        if (v) atomicAdd(&(&c->hist[0][0])[i], v);
    }
}

void launch_keys(const float4* pos, int n, bh_dev_ctrl* ctrl, void* keys, int curve, bool deep, int grid,
                 cudaStream_t s)
{
    if (deep) {
        bh_key64* k = (bh_key64*)keys;
        if (curve == BH_CURVE_HILBERT) bh_keys_kernel<BH_CURVE_HILBERT, bh_key64><<<grid, 256, 0, s>>>(pos, n, ctrl, k);
        else bh_keys_kernel<BH_CURVE_MORTON, bh_key64><<<grid, 256, 0, s>>>(pos, n, ctrl, k);
    } else {
        uint32_t* k = (uint32_t*)keys;
        if (curve == BH_CURVE_HILBERT) bh_keys_kernel<BH_CURVE_HILBERT, uint32_t><<<grid, 256, 0, s>>>(pos, n, ctrl, k);
        else bh_keys_kernel<BH_CURVE_MORTON, uint32_t><<<grid, 256, 0, s>>>(pos, n, ctrl, k);
    }
}

// ------------------------------------------------------------- onesweep
// Look-back status word: epoch (32 bits) | flag (2 bits) | value (30 bits).
// flag 1 = tile aggregate only, 2 = inclusive prefix.  The epoch changes at
// every pass, so stale words from earlier passes read as "not ready" and the
// array never needs clearing.  It is derived on the device from the control
// block's build counter (advanced by bh_init_kernel at every build), never
// passed from the host: a build replayed from a CUDA graph still gets epochs
// that no earlier execution wrote.
constexpr unsigned int kFlagAgg = 1u, kFlagPrefix = 2u;
constexpr int kSpinLimit = 1 << 22;

// Wait until the look-back word at q belongs to this pass (epoch) and carries
// a flag.  False after kSpinLimit polls or once another block has aborted.
__device__ __forceinline__ bool bh_lookback_wait(const volatile unsigned long long* q, unsigned int epoch,
                                                 const bh_dev_ctrl* c, unsigned long long& st)
{
    st = *q;
    int spins = 0;
    while ((unsigned int)(st >> 32) != epoch || ((st >> 30) & 3ull) == 0ull) {
        if (++spins > kSpinLimit || *(const volatile unsigned int*)&c->abort) return false;
        __nanosleep(32);
        st = *q;
    }
    return true;
}

__device__ __forceinline__ bool bh_lookback_ready(unsigned long long st, unsigned int epoch)
{
    return (unsigned int)(st >> 32) == epoch && ((st >> 30) & 3ull) != 0ull;
}

__device__ __forceinline__ unsigned long long bh_status_word(unsigned int epoch, unsigned int flag, unsigned int v)
{
    return ((unsigned long long)epoch << 32) | ((unsigned long long)flag << 30) | (unsigned long long)(v & 0x3fffffffu);
}

// Exclusive scan over the block's first 256 threads (one value each; the
// other threads pass 0 and get 0).  Every thread of the block calls it.
__device__ __forceinline__ unsigned int bh_block_excl_scan256(unsigned int v, unsigned int* warp_tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(BH_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (w < 8 && lane == 31) warp_tot[w] = incl;
    __syncthreads();
    unsigned int base = 0;
    if (w < 8)
        for (int i = 0; i < w; i++) base += warp_tot[i];
    __syncthreads();
    return w < 8 ? base + incl - v : 0u;
}

// Sum of the tile aggregates before `tile` for digit d, down to the nearest
// inclusive prefix (decoupled look-back).  kLookbackBatch predecessors are
// read at once; the first one not yet published is waited for (bounded).
__device__ __forceinline__ bool bh_lookback(const unsigned long long* lookback, int tile, int d, unsigned int epoch,
                                            const bh_dev_ctrl* c, unsigned int& prefix)
{
    prefix = 0u;
    int j = tile - 1;
    while (j >= 0) {
        unsigned long long st[kLookbackBatch];
#pragma unroll
        for (int u = 0; u < kLookbackBatch; u++)
            st[u] = j - u >= 0 ? *((const volatile unsigned long long*)lookback + (size_t)(j - u) * 256 + d) : 0ull;
        int used = 0;
        bool stop = false;
#pragma unroll
        for (int u = 0; u < kLookbackBatch; u++) {
            if (stop || j - u < 0 || !bh_lookback_ready(st[u], epoch)) {
                stop = true;
                continue;
            }
            prefix += (unsigned int)(st[u] & 0x3fffffffull);
            used = u + 1;
            if (((st[u] >> 30) & 3ull) == kFlagPrefix) return true;
        }
        j -= used;
        if (j < 0) return true;
        if (used < kLookbackBatch) {  // word j is not published yet
            unsigned long long w;
            if (!bh_lookback_wait((const volatile unsigned long long*)lookback + (size_t)j * 256 + d, epoch, c, w))
                return false;
            prefix += (unsigned int)(w & 0x3fffffffull);
            if (((w >> 30) & 3ull) == kFlagPrefix) return true;
            j--;
        }
    }
    return true;
}

// One onesweep pass over a tile of TILE keys (4096 30-bit keys, or 2048
// 63-bit keys so that the tile fits the static shared memory) by THREADS
// threads, ITEMS = TILE / THREADS keys per thread.
template <typename K, int TILE, int THREADS, bool FIRST, bool LAST>
__global__ void __launch_bounds__(THREADS)
bh_onesweep_kernel(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
                   uint32_t* __restrict__ vout, const float4* __restrict__ pos, float4* __restrict__ pos_s, int n,
                   int shift, int pass, unsigned long long* lookback, bh_dev_ctrl* c)
{
    const unsigned int epoch = c->build_seq * 8u + (unsigned int)pass + 1u;
    constexpr int W = THREADS / 32;
    constexpr int ITEMS = TILE / THREADS;
    static_assert(ITEMS * THREADS == TILE && THREADS >= 256, "tile shape");
    __shared__ K s_keys[TILE];
    __shared__ uint32_t s_vals[TILE];
    __shared__ unsigned short s_whist[W][256];  // per warp and digit: counts, then offsets (< TILE)
    __shared__ unsigned int s_start[256];  // tile-local start of each digit
    __shared__ int s_base[256];            // global position of a digit's first tile-local slot
    __shared__ unsigned int s_wtot[8];
    __shared__ int s_tile;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) s_tile = (int)atomicAdd(&c->tile_ctr[pass], 1u);
    for (int i = tid; i < W * 256; i += THREADS) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const int tile = s_tile;
    const int base = tile * TILE;
    if (base >= n) return;
    const int tile_n = min(TILE, n - base);

    // warp-striped load: item k of lane l of warp w is tile position w*32*ITEMS + k*32 + l
    K key[ITEMS];
    uint32_t val[ITEMS], rank[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        const int p = base + w * (32 * ITEMS) + k * 32 + lane;
        const bool ok = p < n;
        key[k] = ok ? kin[p] : ~(K)0;
        val[k] = FIRST ? (uint32_t)p : (ok ? vin[p] : 0u);
    }
    // peers of every item first (independent), then the stable rank within
    // the warp, item by item: earlier items, then lower lanes of this item
    const unsigned int lt = bh_lanemask_lt();
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        const bool ok = base + w * (32 * ITEMS) + k * 32 + lane < n;
        const unsigned int d = ok ? ((unsigned int)(key[k] >> shift) & 255u) : 256u;
        rank[k] = __match_any_sync(BH_FULL_MASK, d);
    }
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        const bool ok = base + w * (32 * ITEMS) + k * 32 + lane < n;
        const unsigned int d = (unsigned int)(key[k] >> shift) & 255u;
        const unsigned int peers = rank[k];
        unsigned int prior = 0u;
        if (ok) prior = s_whist[w][d];
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) s_whist[w][d] = (unsigned short)(prior + __popc(peers));
        __syncwarp();
        rank[k] = prior + __popc(peers & lt);
    }
    __syncthreads();

    // per digit (thread = digit): exclusive over warps, tile count
    const int d = tid;
    unsigned int tile_cnt = 0u;
    if (d < 256) {
#pragma unroll
        for (int i = 0; i < W; i++) {
            const unsigned int t = s_whist[i][d];
            s_whist[i][d] = (unsigned short)tile_cnt;
            tile_cnt += t;
        }
        unsigned long long* my = lookback + (size_t)tile * 256 + d;
        *(volatile unsigned long long*)my = bh_status_word(epoch, tile == 0 ? kFlagPrefix : kFlagAgg, tile_cnt);
    }
    const unsigned int tstart = bh_block_excl_scan256(tile_cnt, s_wtot);
    const unsigned int goff = bh_block_excl_scan256(d < 256 ? c->hist[pass][d] : 0u, s_wtot);

    // decoupled look-back over earlier tiles (bounded waits)
    if (d < 256) {
        unsigned int prefix = 0u;
        if (tile > 0) {
            if (!bh_lookback(lookback, tile, d, epoch, c, prefix)) bh_set_error(c, BH_ERR_DEVICE_TIMEOUT);
            *(volatile unsigned long long*)(lookback + (size_t)tile * 256 + d) =
                bh_status_word(epoch, kFlagPrefix, prefix + tile_cnt);
        }
        s_start[d] = tstart;
        s_base[d] = (int)(goff + prefix) - (int)tstart;
    }
    __syncthreads();

    // scatter into shared memory in sorted order
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        const int p = base + w * (32 * ITEMS) + k * 32 + lane;
        if (p < n) {
            const unsigned int dg = (unsigned int)(key[k] >> shift) & 255u;
            const unsigned int sp = s_start[dg] + s_whist[w][dg] + rank[k];
            s_keys[sp] = key[k];
            s_vals[sp] = val[k];
        }
    }
    __syncthreads();
    // write out: runs of equal digits go to consecutive global positions;
    // every load of a thread (the particle gathers of the last pass among
    // them) is issued before its first store
    int dst[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; k++) {
        const int i = tid + k * THREADS;
        dst[k] = -1;
        if (i < tile_n) {
            key[k] = s_keys[i];
            val[k] = s_vals[i];
            const int dd = s_base[(unsigned int)(key[k] >> shift) & 255u] + i;
            if (dd >= 0 && dd < n) dst[k] = dd;
        }
    }
    if (LAST) {
        float4 pv[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; k++)
            if (dst[k] >= 0) pv[k] = pos[val[k] < (uint32_t)n ? val[k] : 0u];
#pragma unroll
        for (int k = 0; k < ITEMS; k++)
            if (dst[k] >= 0) pos_s[dst[k]] = pv[k];
    }
#pragma unroll
    for (int k = 0; k < ITEMS; k++)
        if (dst[k] >= 0) {
            kout[dst[k]] = key[k];
            vout[dst[k]] = val[k];
        }
}

// Passes of 8 bits from the lowest (4 for 30-bit keys, 8 for 63-bit keys;
// an even count, so keys/vals end where they started); the last pass also
// gathers the particles.  vals[k] = caller index of the k-th particle in key order.
// THREADS0: block size of pass 0 (keys only: fewer registers per key).
template <typename K, int TILE, int THREADS0, int THREADS>
static void bh_sort_passes(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt, const float4* pos,
                           float4* pos_s, int n, unsigned long long* lookback, bh_dev_ctrl* ctrl, cudaStream_t s)
{
    constexpr int NP = bh_key_traits<K>::kPasses;
    const int tiles = (n + TILE - 1) / TILE;
    K *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < NP; p++) {
        if (p == 0)
            bh_onesweep_kernel<K, TILE, THREADS0, true, false>
                <<<tiles, THREADS0, 0, s>>>(ka, nullptr, kb, vb, pos, pos_s, n, 0, 0, lookback, ctrl);
        else if (p == NP - 1)
            bh_onesweep_kernel<K, TILE, THREADS, false, true>
                <<<tiles, THREADS, 0, s>>>(ka, va, kb, vb, pos, pos_s, n, 8 * p, p, lookback, ctrl);
        else
            bh_onesweep_kernel<K, TILE, THREADS, false, false>
                <<<tiles, THREADS, 0, s>>>(ka, va, kb, vb, pos, pos_s, n, 8 * p, p, lookback, ctrl);
        K* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
}

void launch_sort(void* keys, void* keys_alt, uint32_t* vals, uint32_t* vals_alt, const float4* pos, float4* pos_s,
                 int n, unsigned long long* lookback, bh_dev_ctrl* ctrl, bool deep, cudaStream_t s)
{
    if (n <= 0) return;
    if (deep)
        bh_sort_passes<bh_key64, kSortTileDeep, kSortThreadsDeep, kSortThreadsDeep>(
            (bh_key64*)keys, (bh_key64*)keys_alt, vals, vals_alt, pos, pos_s, n, lookback, ctrl, s);
    else
        bh_sort_passes<uint32_t, kSortTile, kSortThreadsFirst, kSortThreads>(
            (uint32_t*)keys, (uint32_t*)keys_alt, vals, vals_alt, pos, pos_s, n, lookback, ctrl, s);
}

// Self-test of the failure path: one look-back wait on a word that no block
// will ever publish.  It gives up after kSpinLimit polls and records
// BH_ERR_DEVICE_TIMEOUT, as the sort pass would.
__global__ void bh_selftest_lookback_kernel(bh_dev_ctrl* c)
{
    __shared__ unsigned long long word;
    word = 0ull;  // epoch 0, no flag
    __syncthreads();
    unsigned long long st;
    if (!bh_lookback_wait(&word, 1u, c, st)) bh_set_error(c, BH_ERR_DEVICE_TIMEOUT);
}

void launch_selftest_lookback(bh_dev_ctrl* c, cudaStream_t s)
{
    bh_selftest_lookback_kernel<<<1, 32, 0, s>>>(c);
}

}  // namespace bh

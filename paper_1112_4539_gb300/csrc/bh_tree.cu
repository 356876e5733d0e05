// bh_tree.cu -- octree over Morton-sorted keys, cell moments, walk groups.
//
// Sec. 4.1 builds the octree by recursive subdivision of the root cube; here
// the same tree is read off the sorted keys in parallel (keys of L = 10 or
// 21 levels).  For sorted position k let d_k be the deepest level whose cell
// holds both particles k-1 and k (-1 for k = 0): the cells starting at k are
// those of levels d_k+1 .. L.
// A level-l cell is a node iff its parent cell holds more than n_leaf
// particles; a window of n_leaf+1 consecutive particles shares a level-l cell
// iff its end keys share their top 3l bits, so with W_k = the largest such
// shared level over the windows containing k, the nodes containing k are the
// levels 0 .. lambda_k = min(L, W_k + 1), the deepest being k's leaf.  Node
// (k, l) therefore exists for d_k < l <= lambda_k.  Breadth-first order
// (level, then first particle) gives each node its index by a per-level rank.
//
// Sec. 4.4 (host steps 2-3 of the paper's flow) computes the cell mass,
// centre of mass and effective size S_eff = (l/theta + s)^2 (Eq. 2); here a
// bottom-up pass per level, leaves from their particles, internal nodes from
// their (contiguous) children, FP64 for nodes above a particle-count
// threshold.
#include "bh_internal.cuh"

namespace bh {

constexpr int kLvlThreads = 256;
constexpr int kLvlPer = kLevelTile / kLvlThreads;  // 8 positions per thread
constexpr int kMaxLeaf = 64;
constexpr int kLeafFp64 = 32;
#ifndef BH_WARP_MOMENT_LEVELS
#define BH_WARP_MOMENT_LEVELS 4
#endif
constexpr int kWarpMomentLevels = BH_WARP_MOMENT_LEVELS;  // levels 0..this: a warp per node, below a thread

// ------------------------------------------------------------ pass 1
// dl[k] = (d_k + 1) | (lambda_k << 5); per-block node counts per level.
// With several independent systems (sys = system of each Morton position,
// systems contiguous), particles of different systems share no cell: a
// system's first particle starts a root, and windows never span systems.
template <typename K>
__global__ void __launch_bounds__(kLvlThreads)
bh_levels_kernel(const K* __restrict__ keys, const uint32_t* __restrict__ sys, int n, int n_leaf,
                 uint16_t* __restrict__ dl, uint32_t* __restrict__ blk_lvl, int nblk)
{
    constexpr int L = bh_key_traits<K>::kMaxLevel;
    __shared__ K sk[kLevelTile + 2 * kMaxLeaf + 2];
    __shared__ uint32_t ss[kLevelTile + 2 * kMaxLeaf + 2];
    __shared__ int8_t sw[kLevelTile + kMaxLeaf + 1];
    __shared__ unsigned int sblk[L + 1];  // the block's node count per level
    const int tid = threadIdx.x;
    const int base = blockIdx.x * kLevelTile;
    if (tid <= L) sblk[tid] = 0u;
    const int lo = base - n_leaf - 1;
    const int span = kLevelTile + 2 * n_leaf + 1;
    for (int i = tid; i < span; i += kLvlThreads) {
        const int p = lo + i;
        const bool in = p >= 0 && p < n;
        sk[i] = in ? keys[p] : (K)0;
        ss[i] = (in && sys) ? sys[p] : 0u;
    }
    __syncthreads();
    // w_j for j in [base - n_leaf, base + kLevelTile): common level of the window [j, j + n_leaf]
    for (int i = tid; i < kLevelTile + n_leaf; i += kLvlThreads) {
        const int j = base - n_leaf + i;
        int wv = -1;
        if (j >= 0 && j + n_leaf < n && ss[j - lo] == ss[j + n_leaf - lo])
            wv = bh_common_level(sk[j - lo], sk[j + n_leaf - lo]);
        sw[i] = (int8_t)wv;
    }
    __syncthreads();
    // W_k = max of w_j over j in [k - n_leaf, k], i.e. sw[k - base .. k - base + n_leaf]
    // (entries for j < 0 hold -1).  A thread's positions k0 + r (r < kLvlPer)
    // share the core sw[t0 + kLvlPer - 1 .. t0 + n_leaf] when n_leaf >= kLvlPer - 1;
    // the rest of window r is a suffix of sw[t0 .. t0 + kLvlPer - 2] and a
    // prefix of sw[t0 + n_leaf + 1 ..] (the same maxima, fewer loads).
    const int t0 = tid * kLvlPer;
    int Wr[kLvlPer];
    if (n_leaf >= kLvlPer - 1) {
        int core = -1;
        for (int i = t0 + kLvlPer - 1; i <= t0 + n_leaf; i++) core = max(core, (int)sw[i]);
        int suf = -1;
#pragma unroll
        for (int r = kLvlPer - 1; r >= 0; r--) {
            if (r < kLvlPer - 1) suf = max(suf, (int)sw[t0 + r]);
            Wr[r] = max(core, suf);
        }
        int pre = -1;
#pragma unroll
        for (int r = 1; r < kLvlPer; r++) {
            pre = max(pre, (int)sw[t0 + n_leaf + r]);
            Wr[r] = max(Wr[r], pre);
        }
    } else {
#pragma unroll
        for (int r = 0; r < kLvlPer; r++) {
            int W = -1;
            for (int i = t0 + r; i <= t0 + r + n_leaf; i++) W = max(W, (int)sw[i]);
            Wr[r] = W;
        }
    }
#pragma unroll
    for (int r = 0; r < kLvlPer; r++) {
        const int k = base + t0 + r;
        if (k >= n) break;
        const int d = (k == 0 || ss[k - 1 - lo] != ss[k - lo]) ? -1 : bh_common_level(sk[k - 1 - lo], sk[k - lo]);
        const int lam = min(L, Wr[r] + 1);
        dl[k] = (uint16_t)((d + 1) | (lam << 5));
        for (int l = d + 1; l <= lam; l++) atomicAdd(&sblk[l], 1u);  // the nodes starting at k (usually none)
    }
    __syncthreads();
    if (tid <= L) blk_lvl[(size_t)tid * nblk + blockIdx.x] = sblk[tid];
}

// 1024-thread block: exclusive scan of v (one per thread), returns the total.
__device__ unsigned int bh_block_scan1024(unsigned int& v, unsigned int* wtot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(BH_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[w] = incl;
    __syncthreads();
    if (w == 0) {
        unsigned int x = (lane < (int)(blockDim.x >> 5)) ? wtot[lane] : 0u;
        unsigned int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(BH_FULL_MASK, xi, o);
            if (lane >= o) xi += t;
        }
        wtot[lane] = xi - x;
        if (lane == 31) wtot[32] = xi;
    }
    __syncthreads();
    const unsigned int total = wtot[32];
    v = wtot[w] + incl - v;
    __syncthreads();
    return total;
}

// In-place exclusive scan of `len` values with one 1024-thread block.
__device__ unsigned int bh_scan_segment(uint32_t* a, int len, unsigned int* wtot)
{
    const int per = (len + 1023) / 1024;
    const int b0 = threadIdx.x * per;
    unsigned int s = 0u;
    for (int i = 0; i < per; i++)
        if (b0 + i < len) s += a[b0 + i];
    unsigned int ex = s;
    const unsigned int total = bh_block_scan1024(ex, wtot);
    unsigned int run = ex;
    for (int i = 0; i < per; i++)
        if (b0 + i < len) {
            const unsigned int t = a[b0 + i];
            a[b0 + i] = run;
            run += t;
        }
    __syncthreads();
    return total;
}

// ------------------------------------------------------------ pass 2
// One block per level (nlev = deepest level + 1 blocks) scans that level's
// per-block node counts; the block that finishes last turns the level totals
// into level offsets.  level_offset[l] for l >= nlev holds the node count.
__global__ void __launch_bounds__(1024) bh_level_scan_kernel(uint32_t* blk_lvl, int nblk, int nlev, bh_dev_ctrl* c,
                                                             long long node_cap)
{
    __shared__ unsigned int wtot[33];
    __shared__ bool last;
    const int l = blockIdx.x;
    const unsigned int t = bh_scan_segment(blk_lvl + (size_t)l * nblk, nblk, wtot);
    if (threadIdx.x == 0) {
        c->level_total[l] = t;
        __threadfence();
        last = atomicAdd(&c->scan_done, 1u) == (unsigned int)(nlev - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const volatile unsigned int* tot = c->level_total;
    unsigned long long run = 0ull;
    for (int k = 0; k < nlev; k++) {
        c->level_offset[k] = (unsigned int)run;
        run += tot[k];
    }
    if ((long long)run > node_cap) {
        bh_set_error(c, BH_ERR_CAPACITY);
        run = 0ull;  // later kernels see an empty tree
        for (int k = 0; k < nlev; k++) c->level_offset[k] = 0u;
    }
    for (int k = nlev; k < BH_LEVEL_SLOTS; k++) c->level_offset[k] = (unsigned int)run;
    c->n_nodes = (unsigned int)run;
}

// ------------------------------------------------------------ pass 3
// Write (first, level, child) of every node at its breadth-first index.
// Position k starts the nodes of levels d_k+1 .. lambda_k (usually none): the
// per-level counts and running indices of a thread live in its own column of
// shared memory, so counting and writing loop over those levels only.
template <int L>
__global__ void __launch_bounds__(kLvlThreads)
bh_node_write_kernel(const uint16_t* __restrict__ dl, int n, const uint32_t* __restrict__ blk_lvl, int nblk,
                     const bh_dev_ctrl* __restrict__ c, int32_t* __restrict__ nfirst, uint8_t* __restrict__ nlevel,
                     int32_t* __restrict__ nchildidx)
{
    __shared__ unsigned int swt[kLvlThreads / 32][L + 1];
    __shared__ unsigned int sx[L + 1][kLvlThreads];  // per level and thread: count, then next node index
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int base = blockIdx.x * kLevelTile;
    if (c->n_nodes == 0u) return;  // capacity error (or empty)
#pragma unroll
    for (int l = 0; l <= L; l++) sx[l][tid] = 0u;
    uint16_t my[kLvlPer];
#pragma unroll
    for (int r = 0; r < kLvlPer; r++) {
        const int k = base + tid * kLvlPer + r;
        my[r] = (k < n) ? dl[k] : (uint16_t)(L + 1);  // d+1 = L+1 > lambda = 0: no node
        const int d = (int)(my[r] & 31) - 1, lam = my[r] >> 5;
        for (int l = d + 1; l <= lam; l++) sx[l][tid]++;
    }
    // per-level exclusive scan over the block (thread order = position order)
#pragma unroll
    for (int l = 0; l <= L; l++) {
        const unsigned int cnt = sx[l][tid];
        unsigned int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int t = __shfl_up_sync(BH_FULL_MASK, incl, o);
            if (lane >= o) incl += t;
        }
        sx[l][tid] = incl - cnt;
        if (lane == 31) swt[w][l] = incl;
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l <= L; l++) {
        unsigned int b = c->level_offset[l] + blk_lvl[(size_t)l * nblk + blockIdx.x];
        for (int i = 0; i < w; i++) b += swt[i][l];
        sx[l][tid] += b;
    }
#pragma unroll
    for (int r = 0; r < kLvlPer; r++) {
        const int k = base + tid * kLvlPer + r;
        const int d = (int)(my[r] & 31) - 1, lam = my[r] >> 5;
        int below = -1;  // index of node (k, l+1)
        for (int l = lam; l > d; l--) {
            const int idx = (int)sx[l][tid]++;
            nfirst[idx] = k;
            nlevel[idx] = (uint8_t)l;
            nchildidx[idx] = (l < lam) ? below : -1;
            below = idx;
        }
    }
}

// ------------------------------------------------------------ pass 4
// Particle count of each node (end of its key range by galloping search),
// number of children, packed walk record, leaf statistics.
template <typename K>
__global__ void __launch_bounds__(256)
bh_node_finalize_kernel(const K* __restrict__ keys, const uint32_t* __restrict__ sys,
                        const int32_t* __restrict__ sys_off, int n, bh_nodes nd, bh_dev_ctrl* c)
{
    constexpr int L = bh_key_traits<K>::kMaxLevel;
    const int nn = (int)c->n_nodes;
    unsigned int leaves = 0u, maxleaf = 0u;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
        const int l = nd.level[v];
        const int k = nd.first[v];
        // a node never extends past its system's last particle
        const int seg_end = sys ? sys_off[sys[k] + 1] : n;
        int end = seg_end;
        if (l > 0) {
            const int sh = 3 * (L - l);
            const K target = ((keys[k] >> sh) + (K)1) << sh;
            int lo = k, hi = k + 1, step = 1;
            while (hi < seg_end && keys[hi] < target) {
                lo = hi;
                step <<= 1;
                hi = k + step;
            }
            if (hi > seg_end) hi = seg_end;
            while (hi - lo > 1) {
                const int mid = lo + ((hi - lo) >> 1);
                if (keys[mid] < target) lo = mid;
                else hi = mid;
            }
            end = hi;
        }
        const int cnt = end - k;
        const int ch = nd.child[v];
        int nch = 0;
        if (ch >= 0) {
            const int lim = (int)c->level_offset[l + 2];
            nch = 1;
            while (nch < 8 && ch + nch < lim && nd.first[ch + nch] < end) nch++;
        } else {
            leaves++;
            maxleaf = max(maxleaf, (unsigned int)cnt);
        }
        nd.count[v] = cnt;
        nd.nchild[v] = nch;
        nd.rec[v] = make_int4(k, cnt, ch, nch);
    }
    leaves = __reduce_add_sync(BH_FULL_MASK, leaves);
    maxleaf = __reduce_max_sync(BH_FULL_MASK, maxleaf);
    if ((threadIdx.x & 31) == 0) {
        if (leaves) atomicAdd(&c->n_leaves, leaves);
        if (maxleaf) atomicMax(&c->max_leaf, maxleaf);
    }
}

template <typename K>
static void bh_tree_t(const K* keys, int n, int n_leaf, uint16_t* dl, uint32_t* blk_lvl, const bh_nodes& nd,
                      int64_t node_cap, bh_dev_ctrl* ctrl, int grid, cudaStream_t s, const uint32_t* sys,
                      const int32_t* sys_off)
{
    constexpr int L = bh_key_traits<K>::kMaxLevel;
    const int nblk = (n + kLevelTile - 1) / kLevelTile;
    bh_levels_kernel<K><<<nblk, kLvlThreads, 0, s>>>(keys, sys, n, n_leaf, dl, blk_lvl, nblk);
    bh_level_scan_kernel<<<L + 1, 1024, 0, s>>>(blk_lvl, nblk, L + 1, ctrl, (long long)node_cap);
    bh_node_write_kernel<L><<<nblk, kLvlThreads, 0, s>>>(dl, n, blk_lvl, nblk, ctrl, nd.first, nd.level, nd.child);
    bh_node_finalize_kernel<K><<<grid, 256, 0, s>>>(keys, sys, sys_off, n, nd, ctrl);
}

void launch_tree(const void* keys, bool deep, int n, int n_leaf, uint16_t* dl, uint32_t* blk_lvl, const bh_nodes& nd,
                 int64_t node_cap, bh_dev_ctrl* ctrl, int grid, cudaStream_t s, const uint32_t* sys,
                 const int32_t* sys_off)
{
    if (n <= 0) return;
    if (deep)
        bh_tree_t<bh_key64>((const bh_key64*)keys, n, n_leaf, dl, blk_lvl, nd, node_cap, ctrl, grid, s, sys, sys_off);
    else
        bh_tree_t<uint32_t>((const uint32_t*)keys, n, n_leaf, dl, blk_lvl, nd, node_cap, ctrl, grid, s, sys, sys_off);
}

// ------------------------------------------------------------ groups
// Mark the first particle of every group (see the group rule in the walk
// documentation): children of an internal node holding > G particles are
// packed in octant order into runs of <= G particles; a leaf holding > G
// particles is cut into chunks of G; a root holding <= G is one group.
__global__ void __launch_bounds__(256) bh_group_mark_kernel(bh_nodes nd, int G, uint8_t* __restrict__ flags,
                                                            const bh_dev_ctrl* __restrict__ c)
{
    const int nn = (int)c->n_nodes;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
        const int4 r = nd.rec[v];
        if (v < (int)c->level_offset[1]) {  // a root (one per system)
            if (r.y <= G) flags[r.x] = 1;
            else if (r.z < 0)
                for (int j = 0; j < r.y; j += G) flags[r.x + j] = 1;
        }
        if (r.z < 0 || r.y <= G) continue;
        int run_first = -1, run = 0;
        for (int ci = 0; ci < r.w; ci++) {
            const int4 q = nd.rec[r.z + ci];
            if (q.y <= G) {
                if (run_first >= 0 && run + q.y <= G) {
                    run += q.y;
                } else {
                    if (run_first >= 0) flags[run_first] = 1;
                    run_first = q.x;
                    run = q.y;
                }
            } else {
                if (run_first >= 0) flags[run_first] = 1;
                run_first = -1;
                run = 0;
                if (q.z < 0)
                    for (int j = 0; j < q.y; j += G) flags[q.x + j] = 1;
            }
        }
        if (run_first >= 0) flags[run_first] = 1;
    }
}

constexpr int kFlagThreads = 256;
constexpr int kFlagPer = kFlagTile / kFlagThreads;  // 16 bytes per thread

__global__ void __launch_bounds__(kFlagThreads) bh_flag_count_kernel(const uint8_t* __restrict__ flags, int n,
                                                                     uint32_t* __restrict__ blk)
{
    __shared__ unsigned int ws[kFlagThreads / 32];
    const int base = blockIdx.x * kFlagTile + threadIdx.x * kFlagPer;
    unsigned int s = 0u;
    if (base + kFlagPer <= n) {
        const uint4 q = *reinterpret_cast<const uint4*>(flags + base);
        s = __popc(q.x) + __popc(q.y) + __popc(q.z) + __popc(q.w);  // flags are 0/1 bytes
    } else {
        for (int i = base; i < n && i < base + kFlagPer; i++) s += flags[i];
    }
    s = __reduce_add_sync(BH_FULL_MASK, s);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = 0u;
        for (int i = 0; i < kFlagThreads / 32; i++) t += ws[i];
        blk[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) bh_flag_scan_kernel(uint32_t* blk, int nblk, bh_dev_ctrl* c)
{
    __shared__ unsigned int wtot[33];
    const unsigned int t = bh_scan_segment(blk, nblk, wtot);
    if (threadIdx.x == 0) c->n_groups = t;
}

__global__ void __launch_bounds__(kFlagThreads)
bh_flag_write_kernel(const uint8_t* __restrict__ flags, int n, const uint32_t* __restrict__ blk,
                     int32_t* __restrict__ g_first)
{
    __shared__ unsigned int ws[kFlagThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int base = blockIdx.x * kFlagTile + tid * kFlagPer;
    uint8_t f[kFlagPer];
    unsigned int s = 0u;
#pragma unroll
    for (int i = 0; i < kFlagPer; i++) {
        f[i] = (base + i < n) ? flags[base + i] : (uint8_t)0;
        s += f[i];
    }
    unsigned int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int t = __shfl_up_sync(BH_FULL_MASK, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) ws[w] = incl;
    __syncthreads();
    unsigned int idx = blk[blockIdx.x] + incl - s;
    for (int i = 0; i < w; i++) idx += ws[i];
#pragma unroll
    for (int i = 0; i < kFlagPer; i++)
        if (f[i]) g_first[idx++] = base + i;
}

__global__ void __launch_bounds__(256) bh_group_count_kernel(const int32_t* __restrict__ g_first,
                                                             int32_t* __restrict__ g_count, int n,
                                                             const bh_dev_ctrl* __restrict__ c)
{
    const int ng = (int)c->n_groups;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x)
        g_count[g] = ((g + 1 < ng) ? g_first[g + 1] : n) - g_first[g];
}

void launch_groups(const bh_nodes& nd, int n, int G, uint8_t* flags, uint32_t* blk, int32_t* g_first,
                   int32_t* g_count, bh_dev_ctrl* ctrl, int grid, cudaStream_t s)
{
    if (n <= 0) return;
    const int nblk = (n + kFlagTile - 1) / kFlagTile;
    cudaMemsetAsync(flags, 0, (size_t)nblk * kFlagTile, s);
    bh_group_mark_kernel<<<grid, 256, 0, s>>>(nd, G, flags, ctrl);
    bh_flag_count_kernel<<<nblk, kFlagThreads, 0, s>>>(flags, n, blk);
    bh_flag_scan_kernel<<<1, 1024, 0, s>>>(blk, nblk, ctrl);
    bh_flag_write_kernel<<<nblk, kFlagThreads, 0, s>>>(flags, n, blk, g_first);
    bh_group_count_kernel<<<grid, 256, 0, s>>>(g_first, g_count, n, ctrl);
}

// ------------------------------------------------------------ moments
template <typename R>
struct bh_mom {
    R M, cx, cy, cz, q[6];
};

template <typename R, int ORDER>
__device__ __forceinline__ void bh_leaf_moments(const float4* __restrict__ pos_s, int k, int cnt, bh_mom<R>& o,
                                                bool& massless)
{
    const float4 p0 = pos_s[k];
    const R x0 = p0.x, y0 = p0.y, z0 = p0.z;
    R M = 0, sx = 0, sy = 0, sz = 0;
#pragma unroll 4
    for (int j = k; j < k + cnt; j++) {
        const float4 p = pos_s[j];
        const R m = p.w;
        M += m;
        sx += m * ((R)p.x - x0);
        sy += m * ((R)p.y - y0);
        sz += m * ((R)p.z - z0);
    }
    massless = !(M != (R)0);
    o.M = M;
    o.cx = massless ? x0 : x0 + sx / M;
    o.cy = massless ? y0 : y0 + sy / M;
    o.cz = massless ? z0 : z0 + sz / M;
    if (ORDER >= 2) {
        R q0 = 0, q1 = 0, q2 = 0, q3 = 0, q4 = 0, q5 = 0;
#pragma unroll 4
        for (int j = k; j < k + cnt; j++) {
            const float4 p = pos_s[j];
            const R m = p.w;
            const R a = (R)p.x - o.cx, b = (R)p.y - o.cy, e = (R)p.z - o.cz;
            q0 += m * a * a;
            q1 += m * b * b;
            q2 += m * e * e;
            q3 += m * a * b;
            q4 += m * a * e;
            q5 += m * b * e;
        }
        o.q[0] = q0; o.q[1] = q1; o.q[2] = q2; o.q[3] = q3; o.q[4] = q4; o.q[5] = q5;
    }
}

// Nodes whose moments are combined in FP64: those above the particle-count
// threshold; leaves holding more than kLeafFp64 particles (a sequential FP32
// sum of k equal masses is off by up to ~k * 3e-9 relative, 1e-5 at k = 3000);
// and nodes below level 10 (63-bit keys), whose cells are so small that the
// FP32 centre of mass, good to ~6e-8 of the coordinate scale, would leave
// their second moments with a relative error of ~(6e-8 * scale) / side.
__device__ __forceinline__ bool bh_node_fp64(int count, bool leaf, int level, int fp64_threshold)
{
    return count >= fp64_threshold || (leaf && count > kLeafFp64) || level > BH_MAX_LEVEL;
}

__device__ __forceinline__ double bh_warp_sum(double x)
{
    // butterfly: every lane ends with the same sum (IEEE addition commutes)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(BH_FULL_MASK, x, o);
    return x;
}
__device__ __forceinline__ float bh_warp_sumf(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(BH_FULL_MASK, x, o);
    return x;
}

// Leaves holding more than kLeafFp64 particles (oversized leaves at the
// deepest level, or any leaf when n_leaf > 32) need no other node: a whole
// warp takes each one before the level passes, its lanes striding over the
// particles, and stores the FP64 moments; the level kernel then reads them
// as it reads a child's.  Summed by one thread, a leaf of hundreds of
// particles was the tail of the deepest level's launch.
template <int ORDER>
__global__ void __launch_bounds__(256) bh_bigleaf_moments_kernel(const float4* __restrict__ pos_s, bh_nodes nd,
                                                                  const bh_dev_ctrl* __restrict__ c)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const int nn = (int)c->n_nodes;
    // lane l of warp w examines nodes w + nw (l + 32 i): consecutive nodes go to
    // different warps, so the large leaves of a dense knot (adjacent in the
    // node order) spread over the grid instead of queueing in one warp
    for (long long v0 = warp; v0 < nn; v0 += 32ll * nw) {
        const long long vl = v0 + (long long)nw * lane;
        const int v = vl < nn ? (int)vl : -1;
        int4 r = make_int4(0, 0, 0, 0);
        if (v >= 0) r = nd.rec[v];
        unsigned int big = __ballot_sync(BH_FULL_MASK, v >= 0 && r.z < 0 && r.y > kLeafFp64);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1u;
            const int k = __shfl_sync(BH_FULL_MASK, r.x, src), cnt = __shfl_sync(BH_FULL_MASK, r.y, src);
            const int vw = __shfl_sync(BH_FULL_MASK, v, src);
            // FP32 lane partials of at most count/32 terms, summed across the
            // warp; the mass with a Kahan compensation and the centre of mass
            // in FP64.  Offsets are taken from the first particle, so the
            // relative errors (< (count/32 + 5) * 6e-8 of the offset sums and
            // second moments) stay far below what the moment bars allow.
            const float4 p0 = pos_s[k];
            float kM = 0.f, kc = 0.f, psx = 0.f, psy = 0.f, psz = 0.f;
            for (int j = k + lane; j < k + cnt; j += 32) {
                const float4 p = pos_s[j];
                const float y = __fsub_rn(p.w, kc), t = __fadd_rn(kM, y);
                kc = __fsub_rn(__fsub_rn(t, kM), y);
                kM = t;
                psx = fmaf(p.w, p.x - p0.x, psx);
                psy = fmaf(p.w, p.y - p0.y, psy);
                psz = fmaf(p.w, p.z - p0.z, psz);
            }
            const double M = bh_warp_sum((double)kM - (double)kc);
            psx = bh_warp_sumf(psx);
            psy = bh_warp_sumf(psy);
            psz = bh_warp_sumf(psz);
            const bool massless = !(M != 0.0);
            const double x0 = p0.x, y0 = p0.y, z0 = p0.z;
            const double cx = massless ? x0 : x0 + (double)psx / M;
            const double cy = massless ? y0 : y0 + (double)psy / M;
            const double cz = massless ? z0 : z0 + (double)psz / M;
            double q[6] = {0, 0, 0, 0, 0, 0};
            if (ORDER >= 2) {
                // y = x - COM as (x - x0) - (COM - x0), both offsets small
                const float ox = (float)(cx - x0), oy = (float)(cy - y0), oz = (float)(cz - z0);
                float pq[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int j = k + lane; j < k + cnt; j += 32) {
                    const float4 p = pos_s[j];
                    const float a = (p.x - p0.x) - ox, b = (p.y - p0.y) - oy, e = (p.z - p0.z) - oz;
                    const float ma = p.w * a, mb = p.w * b;
                    pq[0] = fmaf(ma, a, pq[0]);
                    pq[1] = fmaf(mb, b, pq[1]);
                    pq[2] = fmaf(p.w * e, e, pq[2]);
                    pq[3] = fmaf(ma, b, pq[3]);
                    pq[4] = fmaf(ma, e, pq[4]);
                    pq[5] = fmaf(mb, e, pq[5]);
                }
#pragma unroll
                for (int i = 0; i < 6; i++) q[i] = (double)bh_warp_sumf(pq[i]);
            }
            if (lane == 0) {
                nd.com64[vw] = bh_double4{cx, cy, cz, M};
                if (ORDER >= 2)
                    for (int i = 0; i < 6; i++) nd.quad64[(size_t)vw * 6 + i] = q[i];
            }
        }
    }
}

template <typename R>
__device__ __forceinline__ void bh_child_moments(const bh_nodes& nd, int cidx, int fp64_threshold, int order,
                                                 bh_mom<R>& o)
{
    const int cc = nd.count[cidx];
    if (sizeof(R) == 8 && bh_node_fp64(cc, nd.child[cidx] < 0, nd.level[cidx], fp64_threshold)) {
        const bh_double4 c = nd.com64[cidx];
        o.cx = (R)c.x; o.cy = (R)c.y; o.cz = (R)c.z; o.M = (R)c.w;
        if (order >= 2)
            for (int i = 0; i < 6; i++) o.q[i] = (R)nd.quad64[(size_t)cidx * 6 + i];
    } else {
        const float4 c = nd.com_m[cidx];
        o.cx = c.x; o.cy = c.y; o.cz = c.z; o.M = c.w;
        if (order >= 2) {
            const float4 a = nd.quad[2 * (size_t)cidx], b = nd.quad[2 * (size_t)cidx + 1];
            o.q[0] = a.x; o.q[1] = a.y; o.q[2] = a.z; o.q[3] = a.w; o.q[4] = b.x; o.q[5] = b.y;
        }
    }
}

// Two passes over the children (centre of mass, then second moments about
// it), each re-reading the children's records: no per-thread copy of the
// children (which lived in local memory and spilled to L2 at full occupancy).
template <typename R, int ORDER>
__device__ __forceinline__ void bh_internal_moments(const bh_nodes& nd, int ch, int nch, int fp64_threshold,
                                                    bh_mom<R>& o, bool& massless)
{
    bh_mom<R> c0;
    bh_child_moments<R>(nd, ch, fp64_threshold, 1, c0);
    const R x0 = c0.cx, y0 = c0.cy, z0 = c0.cz;
    R M = 0, sx = 0, sy = 0, sz = 0;
    for (int i = 0; i < nch; i++) {
        bh_mom<R> cm;
        bh_child_moments<R>(nd, ch + i, fp64_threshold, 1, cm);
        M += cm.M;
        sx += cm.M * (cm.cx - x0);
        sy += cm.M * (cm.cy - y0);
        sz += cm.M * (cm.cz - z0);
    }
    massless = !(M != (R)0);
    o.M = M;
    o.cx = massless ? x0 : x0 + sx / M;
    o.cy = massless ? y0 : y0 + sy / M;
    o.cz = massless ? z0 : z0 + sz / M;
    if (ORDER >= 2) {
        R q[6] = {0, 0, 0, 0, 0, 0};
        for (int i = 0; i < nch; i++) {
            bh_mom<R> cm;
            bh_child_moments<R>(nd, ch + i, fp64_threshold, 2, cm);
            const R a = cm.cx - o.cx, b = cm.cy - o.cy, e = cm.cz - o.cz, m = cm.M;
            q[0] += cm.q[0] + m * a * a;
            q[1] += cm.q[1] + m * b * b;
            q[2] += cm.q[2] + m * e * e;
            q[3] += cm.q[3] + m * a * b;
            q[4] += cm.q[4] + m * a * e;
            q[5] += cm.q[5] + m * b * e;
        }
        for (int i = 0; i < 6; i++) o.q[i] = q[i];
    }
}

// The same sums with a group of W lanes per node (used with W = 32, a warp,
// on the levels near the root: few nodes, mostly FP64; on the deep levels of
// small leaves groups of 8 or 16 lanes were slower than a thread per node):
// lane j of the group takes particles j, j + W, ... of a leaf (at most
// kLeafFp64 = 32; larger leaves come from bh_bigleaf_moments_kernel) or
// child j of an internal node, and the sums are butterfly reductions within
// the group, so each of its lanes ends with the same values.  Offsets from
// the first particle / first child, as in the per-thread form; only the
// order of the additions differs.
// The lanes of this thread's group of W (all of them take the same path: one node).
template <int W>
__device__ __forceinline__ unsigned int bh_group_mask()
{
    return W == 32 ? BH_FULL_MASK : ((1u << W) - 1u) << ((threadIdx.x & 31) & ~(W - 1));
}
template <int W, typename R>
__device__ __forceinline__ R bh_wsum(R x)
{
    const unsigned int mask = bh_group_mask<W>();
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
}

template <int W, typename R, int ORDER>
__device__ __forceinline__ void bh_leaf_moments_warp(const float4* __restrict__ pos_s, int k, int cnt, bh_mom<R>& o,
                                                     bool& massless)
{
    constexpr int NP = 32 / W;  // particles per lane
    const int j = threadIdx.x & (W - 1);
    const float4 p0 = pos_s[k];
    float4 p[NP];
    R m[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) {
        const int jj = j + i * W;
        p[i] = jj < cnt ? pos_s[k + jj] : p0;
        m[i] = jj < cnt ? (R)p[i].w : (R)0;
    }
    const R x0 = p0.x, y0 = p0.y, z0 = p0.z;
    R M = 0, sx = 0, sy = 0, sz = 0;
#pragma unroll
    for (int i = 0; i < NP; i++) {
        M += m[i];
        sx += m[i] * ((R)p[i].x - x0);
        sy += m[i] * ((R)p[i].y - y0);
        sz += m[i] * ((R)p[i].z - z0);
    }
    M = bh_wsum<W>(M);
    sx = bh_wsum<W>(sx);
    sy = bh_wsum<W>(sy);
    sz = bh_wsum<W>(sz);
    massless = !(M != (R)0);
    o.M = M;
    o.cx = massless ? x0 : x0 + sx / M;
    o.cy = massless ? y0 : y0 + sy / M;
    o.cz = massless ? z0 : z0 + sz / M;
    if (ORDER >= 2) {
        R q[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < NP; i++) {
            const R a = (R)p[i].x - o.cx, b = (R)p[i].y - o.cy, e = (R)p[i].z - o.cz;
            q[0] += m[i] * a * a;
            q[1] += m[i] * b * b;
            q[2] += m[i] * e * e;
            q[3] += m[i] * a * b;
            q[4] += m[i] * a * e;
            q[5] += m[i] * b * e;
        }
#pragma unroll
        for (int i = 0; i < 6; i++) o.q[i] = bh_wsum<W>(q[i]);
    }
}

template <int W, typename R, int ORDER>
__device__ __forceinline__ void bh_internal_moments_warp(const bh_nodes& nd, int ch, int nch, int fp64_threshold,
                                                         bh_mom<R>& o, bool& massless)
{
    static_assert(W >= 8, "a lane per child");
    const int j = threadIdx.x & (W - 1);
    const int base = (threadIdx.x & 31) & ~(W - 1);  // the group's first lane
    bh_mom<R> c;
    bh_child_moments<R>(nd, ch + (j < nch ? j : 0), fp64_threshold, ORDER, c);
    const R m = j < nch ? c.M : (R)0;
    const unsigned int mask = bh_group_mask<W>();
    const R x0 = __shfl_sync(mask, c.cx, base), y0 = __shfl_sync(mask, c.cy, base), z0 = __shfl_sync(mask, c.cz, base);
    const R M = bh_wsum<W>(m);
    const R sx = bh_wsum<W>(m * (c.cx - x0)), sy = bh_wsum<W>(m * (c.cy - y0)), sz = bh_wsum<W>(m * (c.cz - z0));
    massless = !(M != (R)0);
    o.M = M;
    o.cx = massless ? x0 : x0 + sx / M;
    o.cy = massless ? y0 : y0 + sy / M;
    o.cz = massless ? z0 : z0 + sz / M;
    if (ORDER >= 2) {
        const R a = c.cx - o.cx, b = c.cy - o.cy, e = c.cz - o.cz;
        const R own = j < nch ? (R)1 : (R)0;
        o.q[0] = bh_wsum<W>(own * c.q[0] + m * a * a);
        o.q[1] = bh_wsum<W>(own * c.q[1] + m * b * b);
        o.q[2] = bh_wsum<W>(own * c.q[2] + m * e * e);
        o.q[3] = bh_wsum<W>(own * c.q[3] + m * a * b);
        o.q[4] = bh_wsum<W>(own * c.q[4] + m * a * e);
        o.q[5] = bh_wsum<W>(own * c.q[5] + m * b * e);
    }
}

// Moments of one node v of level lev (leaves from their particles, internal
// nodes from their children, which the previous, deeper level wrote).
template <int ORDER, typename K, int W>
__device__ __forceinline__ void bh_moment_node(const float4* __restrict__ pos_s, const K* __restrict__ keys,
                                               const bh_nodes& nd, int v, int lev, float theta, int fp64_threshold,
                                               int curve, float4 gbox, const uint32_t* __restrict__ sys,
                                               const float4* __restrict__ sys_box)
{
    constexpr int L = bh_key_traits<K>::kMaxLevel;
    const int4 r = nd.rec[v];
    // root cube of the node's system (several systems: one cube each)
    const float4 bx = sys ? sys_box[sys[r.x]] : gbox;
    const float xmin = bx.x, ymin = bx.y, zmin = bx.z;
    const float side = ldexpf(bx.w, -lev);  // exact: power-of-two scaling
    const float opening = side / theta;
    const bool f64 = bh_node_fp64(r.y, r.z < 0, lev, fp64_threshold);
    // geometric centre of the node's level-lev cell: the ancestor of the
    // first particle's cell, decoded from its key
    unsigned int ix, iy, iz;
    bh_cell_of<K>(keys[r.x], curve, ix, iy, iz);
    const int sh = L - lev;
    const float gx = xmin + ((float)(ix >> sh) + 0.5f) * side;
    const float gy = ymin + ((float)(iy >> sh) + 0.5f) * side;
    const float gz = zmin + ((float)(iz >> sh) + 0.5f) * side;
    float cx, cy, cz, M, q[6];
    bool massless;
    const bool writer = (threadIdx.x & (W - 1)) == 0;  // the lanes of a node's group hold the same sums
    if (f64) {
        bh_mom<double> o;
        if (r.z < 0 && r.y > kLeafFp64) {
            // taken by bh_bigleaf_moments_kernel
            const bh_double4 m4 = nd.com64[v];
            o.cx = m4.x; o.cy = m4.y; o.cz = m4.z; o.M = m4.w;
            massless = !(o.M != 0.0);
            if (ORDER >= 2)
                for (int i = 0; i < 6; i++) o.q[i] = nd.quad64[(size_t)v * 6 + i];
        } else if (r.z < 0) {
            if (W > 1) bh_leaf_moments_warp<(W > 1 ? W : 8), double, ORDER>(pos_s, r.x, r.y, o, massless);
            else bh_leaf_moments<double, ORDER>(pos_s, r.x, r.y, o, massless);
        } else {
            if (W > 1) bh_internal_moments_warp<(W > 1 ? W : 8), double, ORDER>(nd, r.z, r.w, fp64_threshold, o, massless);
            else bh_internal_moments<double, ORDER>(nd, r.z, r.w, fp64_threshold, o, massless);
        }
        if (massless) {
            o.cx = gx; o.cy = gy; o.cz = gz;
        }
        if (writer) nd.com64[v] = bh_double4{o.cx, o.cy, o.cz, o.M};
        cx = (float)o.cx; cy = (float)o.cy; cz = (float)o.cz; M = (float)o.M;
        if (ORDER >= 2)
            for (int i = 0; i < 6; i++) {
                if (writer) nd.quad64[(size_t)v * 6 + i] = o.q[i];
                q[i] = (float)o.q[i];
            }
    } else {
        bh_mom<float> o;
        if (r.z < 0) {
            if (W > 1) bh_leaf_moments_warp<(W > 1 ? W : 8), float, ORDER>(pos_s, r.x, r.y, o, massless);
            else bh_leaf_moments<float, ORDER>(pos_s, r.x, r.y, o, massless);
        } else {
            if (W > 1) bh_internal_moments_warp<(W > 1 ? W : 8), float, ORDER>(nd, r.z, r.w, fp64_threshold, o, massless);
            else bh_internal_moments<float, ORDER>(nd, r.z, r.w, fp64_threshold, o, massless);
        }
        if (massless) {
            o.cx = gx; o.cy = gy; o.cz = gz;
        }
        cx = o.cx; cy = o.cy; cz = o.cz; M = o.M;
        if (ORDER >= 2)
            for (int i = 0; i < 6; i++) q[i] = o.q[i];
    }
    if (!writer) return;
    nd.com_m[v] = make_float4(cx, cy, cz, M);
    const float dx = gx - cx, dy = gy - cy, dz = gz - cz;
    const float s = sqrtf(dx * dx + dy * dy + dz * dz);
    const float t = opening + s;
    nd.seff[v] = t * t;
    float4 qa = make_float4(0.f, 0.f, 0.f, 0.f), qb = qa;
    if (ORDER >= 2) {
        const float T = q[0] + q[1] + q[2];
        qa = make_float4(q[0], q[1], q[2], q[3]);
        qb = make_float4(q[4], q[5], 1.5f * T, 0.5f * T);
        nd.quad[2 * (size_t)v] = qa;
        nd.quad[2 * (size_t)v + 1] = qb;
    }
    if (nd.wrec) {
        float4* w = nd.wrec + (size_t)v * bh_wrec_f4(ORDER);
        const int chn = r.z < 0 ? -1 : (r.z << 3) | (r.w - 1);
        w[0] = make_float4(cx, cy, cz, M);
        w[1] = make_float4(__int_as_float(r.x), __int_as_float(r.y), __int_as_float(chn), t * t);
        if (ORDER >= 2) {
            w[2] = qa;
            w[3] = qb;
        }
    }
}

// One launch per level, deepest first, W lanes per node: 32 on the levels near
// the root (kWarpMomentLevels: few nodes, FP64 sums whose dependent chains a
// warp shortens to a few reductions), 1 below (4 blocks per SM, at most 64
// registers: the deep levels are bound by the latency of their loads).
template <int ORDER, typename K, int W>
__global__ void __launch_bounds__(256, W == 32 ? 1 : 4)
bh_moments_level_kernel(const float4* __restrict__ pos_s, const K* __restrict__ keys, bh_nodes nd, int lev,
                        float theta, int fp64_threshold, int curve, const bh_dev_ctrl* __restrict__ c,
                        const uint32_t* __restrict__ sys, const float4* __restrict__ sys_box)
{
    const int v0 = (int)c->level_offset[lev], v1 = (int)c->level_offset[lev + 1];
    if (c->n_nodes == 0u) return;
    const float4 gbox = make_float4(c->box[0], c->box[1], c->box[2], c->box[3]);
    // the W lanes of a group share one node per iteration (and so one path)
    const int first = (blockIdx.x * blockDim.x + threadIdx.x) / W, stride = gridDim.x * blockDim.x / W;
    for (int v = v0 + first; v < v1; v += stride)
        bh_moment_node<ORDER, K, W>(pos_s, keys, nd, v, lev, theta, fp64_threshold, curve, gbox, sys, sys_box);
}

template <typename K>
static void bh_moments_t(const float4* pos_s, const K* keys, const bh_nodes& nd, int order, float theta,
                         int fp64_threshold, int curve, bh_dev_ctrl* ctrl, int grid, cudaStream_t s,
                         const uint32_t* sys, const float4* sys_box)
{
    if (order >= 2) bh_bigleaf_moments_kernel<2><<<grid, 256, 0, s>>>(pos_s, nd, ctrl);
    else bh_bigleaf_moments_kernel<1><<<grid, 256, 0, s>>>(pos_s, nd, ctrl);
    for (int lev = bh_key_traits<K>::kMaxLevel; lev >= 0; lev--) {
        const bool warp = lev <= kWarpMomentLevels;
        if (order >= 2) {
            if (warp)
                bh_moments_level_kernel<2, K, 32><<<grid, 256, 0, s>>>(pos_s, keys, nd, lev, theta, fp64_threshold,
                                                                       curve, ctrl, sys, sys_box);
            else
                bh_moments_level_kernel<2, K, 1><<<grid, 256, 0, s>>>(
                    pos_s, keys, nd, lev, theta, fp64_threshold, curve, ctrl, sys, sys_box);
        } else {
            if (warp)
                bh_moments_level_kernel<1, K, 32><<<grid, 256, 0, s>>>(pos_s, keys, nd, lev, theta, fp64_threshold,
                                                                       curve, ctrl, sys, sys_box);
            else
                bh_moments_level_kernel<1, K, 1><<<grid, 256, 0, s>>>(
                    pos_s, keys, nd, lev, theta, fp64_threshold, curve, ctrl, sys, sys_box);
        }
    }
}

void launch_moments(const float4* pos_s, const void* keys, bool deep, const bh_nodes& nd, int order, float theta,
                    int fp64_threshold, int curve, bh_dev_ctrl* ctrl, int grid, cudaStream_t s, const uint32_t* sys,
                    const float4* sys_box)
{
    if (deep)
        bh_moments_t<bh_key64>(pos_s, (const bh_key64*)keys, nd, order, theta, fp64_threshold, curve, ctrl, grid, s,
                               sys, sys_box);
    else
        bh_moments_t<uint32_t>(pos_s, (const uint32_t*)keys, nd, order, theta, fp64_threshold, curve, ctrl, grid, s,
                               sys, sys_box);
}

}  // namespace bh

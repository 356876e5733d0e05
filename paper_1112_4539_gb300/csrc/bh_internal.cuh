// bh_internal.cuh -- device-side layout shared by the kernels of libbhtree.
//
// Everything here belongs to the CUDA library; nothing is shared with the CPU
// oracle.  Tree conventions (Sec. 4.1, Sec. 5 of the paper, with this
// library's readings):
//   * keys of 10 bits per axis (30-bit, uint32) or 21 bits per axis (63-bit,
//     uint64), x in the high bit of each triple, Morton or Peano-Hilbert order;
//   * node = non-empty cell of the 2^l grid (l = 0..L, L = 10 or 21) whose
//     parent cell holds more than n_leaf particles; leaf = holds <= n_leaf
//     particles or l == L;
//   * nodes are stored breadth first (sorted by level, then first particle),
//     so the children of a node are contiguous.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/bhtree.h"

#define BH_MAX_LEVEL 10        // deepest level of 30-bit keys
#define BH_MAX_LEVEL_DEEP 21   // deepest level of 63-bit keys
#define BH_LEVEL_SLOTS 23      // level-indexed arrays: levels 0..21 and the total
#define BH_FULL_MASK 0xffffffffu

// ------------------------------------------------------------------ control
// One control block per context, in device memory.  Reset at every
// tree_build by bh_init_kernel (tree_force resets its own counters).
struct bh_dev_ctrl {
    unsigned int minmax[6];      // ordered-uint encoded min x,y,z then max x,y,z
    float box[4];                // xmin, ymin, zmin, L  (written by the keys kernel)
    float inv;                   // 1024 / L
    unsigned int status;         // first device-side error, as -BH_ERR_* (0 = ok)
    unsigned int abort;          // set with status: waiting kernels give up early
    unsigned int hist[8][256];   // upfront digit histograms of the sort passes (4 or 8)
    unsigned int tile_ctr[8];    // onesweep tile tickets, one per pass
    unsigned int level_total[BH_LEVEL_SLOTS];
    unsigned int level_offset[BH_LEVEL_SLOTS];  // first node of each level; entries past the
                                                // deepest level hold the node count
    unsigned int n_nodes;        // node count of the last build
    unsigned int n_leaves;
    unsigned int max_leaf;
    unsigned int n_groups;
    unsigned int group_ctr;      // walk work queue
    unsigned long long n_pp;
    unsigned long long n_pc;
    unsigned long long cum_pp;   // since context creation (never reset)
    unsigned long long cum_pc;
    unsigned int build_seq;      // builds since the block was zeroed (never reset): the sort
                                 // passes of build b use look-back epochs 8 b + 1 .. 8 b + 8
    unsigned int scan_done;      // level-scan blocks finished (the last one writes the offsets)
    unsigned int pad[6];
};

// Record a device-side error (first one wins) and raise the abort flag.
__device__ __forceinline__ void bh_set_error(bh_dev_ctrl* c, int code)
{
    atomicCAS(&c->status, 0u, (unsigned int)(-code));
    atomicExch(&c->abort, 1u);
}

// Order-preserving map float -> uint (for atomicMin/Max on floats).
__device__ __forceinline__ unsigned int bh_f2ord(float f)
{
    const unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float bh_ord2f(unsigned int u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Key width: 30-bit keys (10 levels, 4 sort passes of 8 bits) or 63-bit keys
// (21 levels, 8 passes).
template <typename K>
struct bh_key_traits;
template <>
struct bh_key_traits<uint32_t> {
    static constexpr int kMaxLevel = BH_MAX_LEVEL;
    static constexpr int kPasses = 4;
};
template <>
struct bh_key_traits<unsigned long long> {
    static constexpr int kMaxLevel = BH_MAX_LEVEL_DEEP;
    static constexpr int kPasses = 8;
};
typedef unsigned long long bh_key64;

// Spread the low 10 bits of v to every third bit (bit k -> bit 3k).
__device__ __forceinline__ unsigned int bh_spread3(unsigned int v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
// Inverse of bh_spread3.
__device__ __forceinline__ unsigned int bh_compact3(unsigned int v)
{
    v &= 0x09249249u;
    v = (v | (v >> 2)) & 0x030c30c3u;
    v = (v | (v >> 4)) & 0x0300f00fu;
    v = (v | (v >> 8)) & 0x030000ffu;
    v = (v | (v >> 16)) & 0x000003ffu;
    return v;
}
// 21-bit versions for 63-bit keys: the same doubling steps on 64-bit words.
__device__ __forceinline__ unsigned long long bh_spread3_21(unsigned int v32)
{
    unsigned long long v = v32 & 0x1fffffu;
    v = (v | (v << 32)) & 0x001f00000000ffffull;
    v = (v | (v << 16)) & 0x001f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}
__device__ __forceinline__ unsigned int bh_compact3_21(unsigned long long v)
{
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v | (v >> 4)) & 0x100f00f00f00f00full;
    v = (v | (v >> 8)) & 0x001f0000ff0000ffull;
    v = (v | (v >> 16)) & 0x001f00000000ffffull;
    v = (v | (v >> 32)) & 0x00000000001fffffull;
    return (unsigned int)v;
}
__device__ __forceinline__ uint32_t bh_spread3_k(unsigned int v, uint32_t) { return bh_spread3(v); }
__device__ __forceinline__ bh_key64 bh_spread3_k(unsigned int v, bh_key64) { return bh_spread3_21(v); }
__device__ __forceinline__ unsigned int bh_compact3_k(uint32_t v) { return bh_compact3(v); }
__device__ __forceinline__ unsigned int bh_compact3_k(bh_key64 v) { return bh_compact3_21(v); }

// Peano-Hilbert index of a cell (B = 10 or 21 bits per axis), the ordering
// Sec. 5 names as better than Morton's.  Skilling's construction
// ("Programming the Hilbert curve", 2004): from the top level down, the bits
// below the level are reflected in x when an axis has the level's bit set,
// else exchanged between x and that axis; the three words are then
// Gray-coded and interleaved as a Morton key (x in the high bit of each triple).
template <typename K>
__device__ __forceinline__ K bh_hilbert3(unsigned int x, unsigned int y, unsigned int z)
{
    constexpr int B = bh_key_traits<K>::kMaxLevel;
#pragma unroll
    for (int lv = B - 1; lv >= 1; lv--) {
        const unsigned int bit = 1u << lv, below = bit - 1u;
        if (x & bit) x ^= below;
        if (y & bit) {
            x ^= below;
        } else {
            const unsigned int d = (x ^ y) & below;
            x ^= d;
            y ^= d;
        }
        if (z & bit) {
            x ^= below;
        } else {
            const unsigned int d = (x ^ z) & below;
            x ^= d;
            z ^= d;
        }
    }
    y ^= x;
    z ^= y;
    unsigned int g = 0u;
#pragma unroll
    for (int lv = B - 1; lv >= 1; lv--)
        if (z & (1u << lv)) g ^= (1u << lv) - 1u;
    x ^= g;
    y ^= g;
    z ^= g;
    return (bh_spread3_k(x, K()) << 2) | (bh_spread3_k(y, K()) << 1) | bh_spread3_k(z, K());
}
// Cell of a Peano-Hilbert index (inverse of bh_hilbert3).
template <typename K>
__device__ __forceinline__ void bh_hilbert3_cell(K h, unsigned int& x, unsigned int& y, unsigned int& z)
{
    constexpr int B = bh_key_traits<K>::kMaxLevel;
    x = bh_compact3_k((K)(h >> 2));
    y = bh_compact3_k((K)(h >> 1));
    z = bh_compact3_k(h);
    const unsigned int g = z >> 1;
    z ^= y;
    y ^= x;
    x ^= g;
#pragma unroll
    for (int lv = 1; lv <= B - 1; lv++) {
        const unsigned int bit = 1u << lv, below = bit - 1u;
        if (z & bit) {
            x ^= below;
        } else {
            const unsigned int d = (x ^ z) & below;
            x ^= d;
            z ^= d;
        }
        if (y & bit) {
            x ^= below;
        } else {
            const unsigned int d = (x ^ y) & below;
            x ^= d;
            y ^= d;
        }
        if (x & bit) x ^= below;
    }
}
// Key of a cell, and cell of a key, for the context's order.
template <int CURVE, typename K>
__device__ __forceinline__ K bh_key_of(unsigned int x, unsigned int y, unsigned int z)
{
    return CURVE == BH_CURVE_HILBERT ? bh_hilbert3<K>(x, y, z)
                                     : (bh_spread3_k(x, K()) << 2) | (bh_spread3_k(y, K()) << 1) |
                                           bh_spread3_k(z, K());
}
template <typename K>
__device__ __forceinline__ void bh_cell_of(K key, int curve, unsigned int& x, unsigned int& y, unsigned int& z)
{
    if (curve == BH_CURVE_HILBERT) {
        bh_hilbert3_cell<K>(key, x, y, z);
    } else {
        x = bh_compact3_k((K)(key >> 2));
        y = bh_compact3_k((K)(key >> 1));
        z = bh_compact3_k(key);
    }
}

// Deepest level whose cell holds both keys (0..L); keys of one cell share
// their top 3*l bits.
__device__ __forceinline__ int bh_common_level(unsigned int a, unsigned int b)
{
    const unsigned int x = a ^ b;
    if (x == 0u) return BH_MAX_LEVEL;
    return (BH_MAX_LEVEL - 1) - (31 - __clz((int)x)) / 3;
}
__device__ __forceinline__ int bh_common_level(unsigned long long a, unsigned long long b)
{
    const unsigned long long x = a ^ b;
    if (x == 0ull) return BH_MAX_LEVEL_DEEP;
    return (BH_MAX_LEVEL_DEEP - 1) - (63 - __clzll((long long)x)) / 3;
}



// Root cube from the reduced bounds (same rule as the build's first kernel).
__device__ __forceinline__ void bh_box_from_minmax(const unsigned int* mm, float* box, float* inv)
{
    const float lo0 = bh_ord2f(mm[0]), lo1 = bh_ord2f(mm[1]), lo2 = bh_ord2f(mm[2]);
    const float hi0 = bh_ord2f(mm[3]), hi1 = bh_ord2f(mm[4]), hi2 = bh_ord2f(mm[5]);
    float L = __fsub_rn(hi0, lo0);
    const float L1 = __fsub_rn(hi1, lo1), L2 = __fsub_rn(hi2, lo2);
    if (L1 > L) L = L1;
    if (L2 > L) L = L2;
    float iv = __fdiv_rn(1024.0f, L);
    if (!(L > 0.0f) || !isfinite(iv)) {
        L = 1.0f;
        iv = 1024.0f;
    }
    box[0] = lo0;
    box[1] = lo1;
    box[2] = lo2;
    box[3] = L;
    *inv = iv;
}

// ---------------------------------------------------------- warp helpers
__device__ __forceinline__ unsigned int bh_lanemask_lt()
{
    unsigned int m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int bh_warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(BH_FULL_MASK, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// 32-byte FP64 vector (x, y, z, w)
struct __align__(32) bh_double4 {
    double x, y, z, w;
};

// ------------------------------------------------------------- node arrays
// Node record read by the walk: first particle, count, first child (-1 for
// leaves), number of children.
struct bh_nodes {
    int32_t* first;
    int32_t* count;
    int32_t* child;
    int32_t* nchild;
    uint8_t* level;
    int4* rec;        // (first, count, child, nchild) packed for the walk
    float4* com_m;    // centre of mass, mass
    float* seff;      // S_eff of Eq. (2)
    float4* quad;     // 2 per node: (xx, yy, zz, xy), (xz, yz, 1.5 T, 0.5 T)
    bh_double4* com64;   // FP64 centre of mass + mass (nodes above the FP64 threshold)
    double* quad64;   // 6 per node (FP64 nodes, order 2)
    // walk records for the TMA-staged walk (nullptr: not kept): one contiguous
    // record per node, so a range of siblings is one bulk copy.  float4 0 =
    // (centre of mass, M); float4 1 = (first, count, child << 3 | (nchild - 1)
    // or -1 for a leaf, S_eff) as bits; order 2 adds the two quad float4s;
    // one float4 of padding makes the record an odd number of float4s, so
    // that 8 lanes reading records i..i+7 from shared memory hit 8 distinct
    // bank quads (no conflicts).
    float4* wrec = nullptr;
};

// float4s per walk record (with its padding)
__host__ __device__ constexpr int bh_wrec_f4(int order) { return order >= 2 ? 5 : 3; }

// --------------------------------------------------------------- launches
// (bodies in the .cu files; all are stream-ordered and take device pointers)
namespace bh {

constexpr int kSortThreads = 512;       // threads of an onesweep block, passes 1-3 (30-bit keys)
constexpr int kSortThreadsFirst = 256;  // threads of pass 0 (30-bit keys: 16 keys per thread)
constexpr int kSortThreadsDeep = 256;   // threads of an onesweep block (63-bit keys)
constexpr int kLookbackBatch = 4;       // predecessors read per look-back step
constexpr int kSortTile = 4096;         // keys per tile (30-bit keys)
constexpr int kSortTileDeep = 2048;     // keys per tile (63-bit keys)
constexpr int kLevelTile = 2048;                       // positions per node-build block
constexpr int kFlagTile = 4096;                        // positions per group-compaction block

void launch_init(bh_dev_ctrl* ctrl, cudaStream_t s);
void launch_bbox(const float4* pos, int n, bh_dev_ctrl* ctrl, int grid, cudaStream_t s);
// keys: uint32_t[n] (30-bit keys) or, with deep, bh_key64[n] (63-bit keys)
void launch_keys(const float4* pos, int n, bh_dev_ctrl* ctrl, void* keys, int curve, bool deep, int grid,
                 cudaStream_t s);
void launch_sort(void* keys, void* keys_alt, uint32_t* vals, uint32_t* vals_alt, const float4* pos, float4* pos_s,
                 int n, unsigned long long* lookback, bh_dev_ctrl* ctrl, bool deep,
                 cudaStream_t s);
// sys / sys_off / sys_box: several independent systems (system of each
// Morton position, first particle of each system + total, root cube of each);
// null for a single system.
// dl: uint16_t[n] scratch; blk_lvl: (deepest level + 1) * ceil(n / kLevelTile) words
void launch_tree(const void* keys, bool deep, int n, int n_leaf, uint16_t* dl, uint32_t* blk_lvl,
                 const bh_nodes& nd, int64_t node_cap, bh_dev_ctrl* ctrl, int grid, cudaStream_t s,
                 const uint32_t* sys = nullptr, const int32_t* sys_off = nullptr);
void launch_groups(const bh_nodes& nd, int n, int G, uint8_t* flags, uint32_t* blk, int32_t* g_first,
                   int32_t* g_count, bh_dev_ctrl* ctrl, int grid, cudaStream_t s);
void launch_moments(const float4* pos_s, const void* keys, bool deep, const bh_nodes& nd, int order,
                    float theta, int fp64_threshold, int curve, bh_dev_ctrl* ctrl, int grid, cudaStream_t s,
                    const uint32_t* sys = nullptr, const float4* sys_box = nullptr);
// One CTA per system: root cube, keys, stable radix sort and gather of each
// system's particles (systems contiguous, each <= kBatchMaxN particles).
constexpr int kBatchMaxN = 65536;
void launch_batch_sort(const float4* pos, const int32_t* sys_off, int nsys, void* keys, void* keys_alt,
                       uint32_t* vals, uint32_t* vals_alt, float4* pos_s, uint32_t* sys, float4* sys_box,
                       int curve, bool deep, bh_dev_ctrl* ctrl, cudaStream_t s);
}  // namespace bh
struct bh_mlp_dev;
namespace bh {
// learned-criterion inputs of the walk (null pointer: plain Eq. 2 criterion)
struct WalkLearned {
    const float4* mfeat;
    const bh_mlp_dev* mlp;
    float theta_guard;
};
int launch_walk(const float4* pos_s, const uint32_t* perm, const int32_t* g_first, const int32_t* g_count,
                const bh_nodes& nd, int order, int G, float eps, float4* out, bh_dev_ctrl* ctrl,
                int sm_count, int block_threads, int blocks_per_sm, cudaStream_t s,
                const WalkLearned* learned = nullptr, int walk_variant = 0);
// failure-path self-tests: one bounded wait that nothing satisfies
void launch_selftest_ring(bh_dev_ctrl* c, cudaStream_t s);
void launch_selftest_tma(bh_dev_ctrl* c, cudaStream_t s);
void launch_selftest_lookback(bh_dev_ctrl* c, cudaStream_t s);
int launch_direct(const float4* src, int n_src, const float4* tgt, const int64_t* self, int n_tgt,
                  double eps, void* out, int precision, cudaStream_t s,
                  const float* eps_src = nullptr, const float* eps_tgt = nullptr);
void launch_kick_drift(float4* pos, float4* vel, const float4* acc, int n, float dt_kick, float dt_drift, int grid,
                       cudaStream_t s);

// kernel launches enqueued by one call of each stage (for bh_stats.launches)
// individual softening: h = eps^2 / 2 per particle (key order) and the mass-weighted mean of h per node
struct bh_soft {
    float* h = nullptr;        // n
    double2* sums = nullptr;   // per node: (sum m, sum m h)
    float* hbar = nullptr;     // per node
};
int launch_pwalk(const float4* pos_s, const uint32_t* perm, const bh_nodes& nd, int32_t* parent, int32_t* next,
                 int order, int n, int node_cap, float eps, bool unsoftened_cells, float4* out, bh_dev_ctrl* ctrl,
                 int sm_count, cudaStream_t s, const bh_soft* soft = nullptr);
void launch_softening(const float* eps, const uint32_t* perm, const float4* pos_s, const bh_nodes& nd, int n,
                      bool deep, const bh_soft& soft, bh_dev_ctrl* ctrl, int grid, cudaStream_t s);

int launch_sph(const float4* pos_s, const uint32_t* perm, const int32_t* g_first, const int32_t* g_count,
               const bh_nodes& nd, float4* blo, float4* bhi, int G, const float* h, float h_const, int32_t* count,
               float* rho, bh_dev_ctrl* ctrl, int sm_count, int grid, int max_level, cudaStream_t s);

// launches per call (deep = 63-bit keys: 8 sort passes, 22 levels)
inline int launches_build(bool deep) { return deep ? 20 : 16; }  // init, bbox, keys, sort passes, 4 tree, 5 groups
inline int launches_moments(bool deep) { return (deep ? 22 : 11) + 1; }  // large leaves, one per level
constexpr int kLaunchesForce = 2;    // counter reset, walk
constexpr int kLaunchesPWalk = 4;    // parent links, next links, counter reset, walk
inline int launches_sph(bool deep) { return (deep ? 22 : 11) + 2; }  // node boxes per level, reset, walk
inline int launches_softening(bool deep) { return (deep ? 22 : 11) + 1; }  // gather, one per level

}  // namespace bh

// bh_batch.cu -- many independent systems in one pass of the build.
//
// Each system (a contiguous range of particles, at most kBatchMaxN) gets its
// own root cube (Sec. 4.1) and key ordering (Sec. 5).  One CTA per system
// does all of it in a single launch: the per-axis bounds, the keys, a stable
// LSD radix sort of the system's (key, index) pairs in 8-bit passes (4 for
// 30-bit keys, 8 for 63-bit keys) over
// global ping-pong buffers (the CTA walks its range tile by tile, ranking each
// tile stably with warp match-any and carrying the running digit offsets, so
// no inter-CTA look-back is needed), and the gather into Morton order.  The
// tree, moments, groups and walk then run over all systems at once.
#include "bh_internal.cuh"

namespace bh {

constexpr int kBT = 512;
constexpr int kBWarps = kBT / 32;
constexpr int kBItems = 8;
constexpr int kBTile = kBT * kBItems;  // 4096 keys per tile

template <typename K>
__global__ void __launch_bounds__(kBT)
bh_batch_sort_kernel(const float4* __restrict__ pos, const int32_t* __restrict__ off, int curve, K* keys,
                     K* keys_alt, uint32_t* vals, uint32_t* vals_alt, float4* __restrict__ pos_s,
                     uint32_t* __restrict__ sys, float4* __restrict__ sys_box, bh_dev_ctrl* c)
{
    constexpr int B = bh_key_traits<K>::kMaxLevel, NP = bh_key_traits<K>::kPasses;
    constexpr unsigned int CMAX = (1u << B) - 1u;
    __shared__ unsigned int whist[kBWarps][256];
    __shared__ unsigned int base[256], run[256], tcnt[256];
    __shared__ unsigned int red[6][kBWarps];
    __shared__ unsigned int wt[8];
    __shared__ float sbox[4];
    __shared__ float sinv;
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int o = off[s], e = off[s + 1];
    if (e <= o) {
        if (tid == 0) sys_box[s] = make_float4(0.f, 0.f, 0.f, 1.f);
        return;
    }
    // ---- root cube (same rule as the single-system build)
    unsigned int lo0 = 0xffffffffu, lo1 = 0xffffffffu, lo2 = 0xffffffffu, hi0 = 0u, hi1 = 0u, hi2 = 0u;
    bool bad = false;
    for (int i = o + tid; i < e; i += kBT) {
        const float4 p = pos[i];
        bad |= !(isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w));
        const unsigned int ox = bh_f2ord(p.x), oy = bh_f2ord(p.y), oz = bh_f2ord(p.z);
        lo0 = min(lo0, ox); lo1 = min(lo1, oy); lo2 = min(lo2, oz);
        hi0 = max(hi0, ox); hi1 = max(hi1, oy); hi2 = max(hi2, oz);
    }
    lo0 = __reduce_min_sync(BH_FULL_MASK, lo0);
    lo1 = __reduce_min_sync(BH_FULL_MASK, lo1);
    lo2 = __reduce_min_sync(BH_FULL_MASK, lo2);
    hi0 = __reduce_max_sync(BH_FULL_MASK, hi0);
    hi1 = __reduce_max_sync(BH_FULL_MASK, hi1);
    hi2 = __reduce_max_sync(BH_FULL_MASK, hi2);
    if (__any_sync(BH_FULL_MASK, bad) && lane == 0) atomicCAS(&c->status, 0u, (unsigned int)(-BH_ERR_NONFINITE));
    if (lane == 0) {
        red[0][w] = lo0; red[1][w] = lo1; red[2][w] = lo2;
        red[3][w] = hi0; red[4][w] = hi1; red[5][w] = hi2;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned int mm[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0u, 0u, 0u};
        for (int i = 0; i < kBWarps; i++) {
            for (int k = 0; k < 3; k++) mm[k] = min(mm[k], red[k][i]);
            for (int k = 3; k < 6; k++) mm[k] = max(mm[k], red[k][i]);
        }
        bh_box_from_minmax(mm, sbox, &sinv);
        sys_box[s] = make_float4(sbox[0], sbox[1], sbox[2], sbox[3]);
    }
    __syncthreads();
    // ---- keys (q = (x - xmin) * (2^B/L), two rounded FP32 ops; c = min(trunc q, 2^B - 1))
    {
        const float x0 = sbox[0], y0 = sbox[1], z0 = sbox[2], inv = __fmul_rn(sinv, (float)(1u << (B - 10)));
        for (int i = o + tid; i < e; i += kBT) {
            const float4 p = pos[i];
            const unsigned int cx = min(__float2uint_rz(__fmul_rn(__fsub_rn(p.x, x0), inv)), CMAX);
            const unsigned int cy = min(__float2uint_rz(__fmul_rn(__fsub_rn(p.y, y0), inv)), CMAX);
            const unsigned int cz = min(__float2uint_rz(__fmul_rn(__fsub_rn(p.z, z0), inv)), CMAX);
            keys[i] = curve == BH_CURVE_HILBERT ? bh_key_of<BH_CURVE_HILBERT, K>(cx, cy, cz)
                                                : bh_key_of<BH_CURVE_MORTON, K>(cx, cy, cz);
            vals[i] = (uint32_t)i;
        }
    }
    __syncthreads();
    // ---- stable 8-bit passes from the lowest bits
    K *sk = keys, *dk = keys_alt;
    uint32_t *sv = vals, *dv = vals_alt;
    const unsigned int lt = bh_lanemask_lt();
    for (int pass = 0; pass < NP; pass++) {
        const int shift = 8 * pass;
        if (tid < 256) base[tid] = 0u;
        __syncthreads();
        for (int i = o + tid; i < e; i += kBT) atomicAdd(&base[(unsigned int)(sk[i] >> shift) & 255u], 1u);
        __syncthreads();
        // exclusive scan of the 256 digit counts (warps 0..7), barrier outside the branch
        unsigned int v = 0u, incl = 0u;
        if (tid < 256) {
            v = base[tid];
            incl = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned int t = __shfl_up_sync(BH_FULL_MASK, incl, d);
                if (lane >= d) incl += t;
            }
            if (lane == 31) wt[w] = incl;
        }
        __syncthreads();
        if (tid < 256) {
            unsigned int add = 0u;
            for (int i = 0; i < w; i++) add += wt[i];
            base[tid] = add + incl - v;
            run[tid] = 0u;
        }
        __syncthreads();
        for (int t0 = o; t0 < e; t0 += kBTile) {
            for (int i = tid; i < kBWarps * 256; i += kBT) (&whist[0][0])[i] = 0u;
            __syncthreads();
            K key[kBItems];
            uint32_t val[kBItems], rank[kBItems];
#pragma unroll
            for (int k = 0; k < kBItems; k++) {
                const int p = t0 + w * (32 * kBItems) + k * 32 + lane;
                const bool ok = p < e;
                key[k] = ok ? sk[p] : (K)0;
                val[k] = ok ? sv[p] : 0u;
                const unsigned int d = ok ? ((unsigned int)(key[k] >> shift) & 255u) : 256u;
                const unsigned int peers = __match_any_sync(BH_FULL_MASK, d);
                unsigned int prior = 0u;
                if (ok) prior = whist[w][d];
                __syncwarp();
                if (ok && lane == __ffs(peers) - 1) whist[w][d] = prior + __popc(peers);
                __syncwarp();
                rank[k] = prior + __popc(peers & lt);
            }
            __syncthreads();
            if (tid < 256) {
                unsigned int r = 0u;
                for (int i = 0; i < kBWarps; i++) {
                    const unsigned int t = whist[i][tid];
                    whist[i][tid] = r;
                    r += t;
                }
                tcnt[tid] = r;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kBItems; k++) {
                const int p = t0 + w * (32 * kBItems) + k * 32 + lane;
                if (p < e) {
                    const unsigned int d = (unsigned int)(key[k] >> shift) & 255u;
                    const int dst = o + (int)(base[d] + run[d] + whist[w][d] + rank[k]);
                    if (dst >= o && dst < e) {
                        dk[dst] = key[k];
                        dv[dst] = val[k];
                    }
                }
            }
            __syncthreads();
            if (tid < 256) run[tid] += tcnt[tid];
            __syncthreads();
        }
        K* tk = sk;
        sk = dk;
        dk = tk;
        uint32_t* t = sv;
        sv = dv;
        dv = t;
        __syncthreads();
    }
    // ---- after an even number of passes the sorted pairs are back in keys / vals
    for (int i = o + tid; i < e; i += kBT) {
        const uint32_t src = sv[i];
        pos_s[i] = pos[(src >= (uint32_t)o && src < (uint32_t)e) ? src : (uint32_t)o];
        sys[i] = (uint32_t)s;
    }
}

void launch_batch_sort(const float4* pos, const int32_t* sys_off, int nsys, void* keys, void* keys_alt,
                       uint32_t* vals, uint32_t* vals_alt, float4* pos_s, uint32_t* sys, float4* sys_box,
                       int curve, bool deep, bh_dev_ctrl* ctrl, cudaStream_t s)
{
    if (nsys <= 0) return;
    if (deep)
        bh_batch_sort_kernel<bh_key64><<<nsys, kBT, 0, s>>>(pos, sys_off, curve, (bh_key64*)keys, (bh_key64*)keys_alt,
                                                            vals, vals_alt, pos_s, sys, sys_box, ctrl);
    else
        bh_batch_sort_kernel<uint32_t><<<nsys, kBT, 0, s>>>(pos, sys_off, curve, (uint32_t*)keys, (uint32_t*)keys_alt,
                                                            vals, vals_alt, pos_s, sys, sys_box, ctrl);
}

}  // namespace bh

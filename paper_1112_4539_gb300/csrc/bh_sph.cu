// bh_sph.cu -- neighbour search and SPH density: the short-range application
// of the general tree walk (Sec. 4.3, Fig. 4).
//
// Fig. 4's walk calls distance_test on each cell and, for a neighbour search,
// skips a cell that lies farther than the search radius (its proc_cell does
// nothing) and descends otherwise; proc_particle tests one pair.  Here, as in
// the gravity walk, one warp walks the tree for a whole group of up to 32*T
// particles: a node is skipped when its particles' bounding box lies farther
// than the group's largest radius from the group's bounding box (with a
// 1e-5 relative allowance, so FP32 rounding of the box gap can never skip a
// neighbour), a leaf contributes all its particles as candidates when its
// box is also within reach of at least one target of the warp (each with its
// own radius), other nodes are opened.  Candidates go through a 64-entry
// ring in shared memory and are tested 32 at a time against each lane's T
// targets.
//
// Pair rule (identical to the oracle's): d = x_j - x_i per axis in FP32,
// r2 = fma(dz, dz, fma(dy, dy, dx * dx)), j != i is a neighbour iff
// r2 < h_i * h_i.  Density rho_i = sum over i and its neighbours of
// m_j W(sqrt(r2), h_i) with the cubic spline of support h (Monaghan &
// Lattanzio 1985), FP32.
#include <algorithm>

#include "bh_internal.cuh"

namespace bh {

#ifndef BH_SPH_LEAF_FILTER
#define BH_SPH_LEAF_FILTER 1
#endif
constexpr int kSphStackCap = 704;   // ranges of <= 8 siblings; same bound as the gravity walk
constexpr int kSphRing = 64;

// ------------------------------------------------------------ node boxes
// Tight bounding box of every node's particles, bottom-up by level: a leaf
// scans its particles, an internal node combines its children (one level
// deeper, already done).  Min/max are exact.
__global__ void bh_node_box_kernel(const float4* __restrict__ pos_s, const int4* __restrict__ rec,
                                   float4* __restrict__ lo, float4* __restrict__ hi, int lev,
                                   const bh_dev_ctrl* __restrict__ c)
{
    const int v0 = (int)c->level_offset[lev], v1 = (int)c->level_offset[lev + 1];
    for (int v = v0 + blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += gridDim.x * blockDim.x) {
        const int4 r = rec[v];
        float4 a = make_float4(INFINITY, INFINITY, INFINITY, 0.f), b = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
        if (r.z < 0) {
            for (int k = r.x; k < r.x + r.y; k++) {
                const float4 p = pos_s[k];
                a.x = fminf(a.x, p.x); a.y = fminf(a.y, p.y); a.z = fminf(a.z, p.z);
                b.x = fmaxf(b.x, p.x); b.y = fmaxf(b.y, p.y); b.z = fmaxf(b.z, p.z);
            }
        } else {
            for (int k = r.z; k < r.z + r.w; k++) {
                const float4 l = lo[k], h = hi[k];
                a.x = fminf(a.x, l.x); a.y = fminf(a.y, l.y); a.z = fminf(a.z, l.z);
                b.x = fmaxf(b.x, h.x); b.y = fmaxf(b.y, h.y); b.z = fmaxf(b.z, h.z);
            }
        }
        lo[v] = a;
        hi[v] = b;
    }
}

// ------------------------------------------------------------ walk
struct SphSmem {
    uint32_t stack[kSphStackCap];
    uint32_t staging[32];
    int2 leafq[64];
    float4 ring[kSphRing];   // candidate particles (x, y, z, m)
    int ridx[kSphRing];      // their Morton positions (self test)
};

struct SphParams {
    const float4* pos_s;
    const uint32_t* perm;
    const int32_t* g_first;
    const int32_t* g_count;
    const int4* rec;
    const float4* blo;
    const float4* bhi;
    const float* h;      // per particle, caller order (nullptr: h_const)
    float h_const;
    int32_t* count;      // caller order (nullptr: not written)
    float* rho;          // caller order (nullptr: not written)
    bh_dev_ctrl* ctrl;
};

// cubic spline with support h (normalised to unit integral), FP32
__device__ __forceinline__ float bh_w3(float r, float hinv, float c)
{
    const float q = r * hinv;
    const float u = 1.0f - q;
    const float inner = fmaf(6.0f * q * q, q - 1.0f, 1.0f);  // 1 - 6 q^2 + 6 q^3
    return c * (q <= 0.5f ? inner : (q <= 1.0f ? 2.0f * u * u * u : 0.0f));
}

template <int T>
__device__ __forceinline__ void bh_sph_tile(const float4* __restrict__ src, const int* __restrict__ sidx, int gb,
                                            const float (&xi)[T], const float (&yi)[T], const float (&zi)[T],
                                            const float (&h2)[T], const float (&hinv)[T], const float (&cw)[T],
                                            int tn, int (&cnt)[T], float (&rho)[T])
{
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < 32; j++) {
        const float4 s = src[j];
        const int js = sidx[j];
#pragma unroll
        for (int t = 0; t < T; t++) {
            if (t < tn) {
                const float dx = __fsub_rn(s.x, xi[t]), dy = __fsub_rn(s.y, yi[t]), dz = __fsub_rn(s.z, zi[t]);
                const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
                const bool self = js == gb + t * 32 + lane;
                if (r2 < h2[t] || self) {
                    cnt[t] += self ? 0 : 1;
                    rho[t] = fmaf(s.w, bh_w3(sqrtf(r2), hinv[t], cw[t]), rho[t]);
                }
            }
        }
    }
}

template <int T>
__global__ void __launch_bounds__(128) bh_sph_kernel(SphParams P)
{
    __shared__ SphSmem smem[4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    SphSmem& S = smem[wib];
    const unsigned int lt = bh_lanemask_lt();
    bh_dev_ctrl* ctrl = P.ctrl;
    const int ng = (int)ctrl->n_groups;
    const int n_roots = (int)ctrl->level_offset[1];
    unsigned long long tested = 0ull;

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&ctrl->group_ctr, 1u);
        g = __shfl_sync(BH_FULL_MASK, g, 0);
        if (g >= ng) break;
        int ab = 0;
        if (lane == 0) ab = (int)*(volatile unsigned int*)&ctrl->abort;
        if (__shfl_sync(BH_FULL_MASK, ab, 0)) break;
        const int gb = P.g_first[g], gc = P.g_count[g];
        const int tn = (gc + 31) >> 5;

        float xi[T], yi[T], zi[T], h2[T], hinv[T], cw[T], rho[T];
        int cnt[T];
        float bx0 = INFINITY, by0 = INFINITY, bz0 = INFINITY, bx1 = -INFINITY, by1 = -INFINITY, bz1 = -INFINITY;
        float hmax = 0.0f;
        bool bad = false;
#pragma unroll
        for (int t = 0; t < T; t++) {
            const int o = t * 32 + lane;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            float h = 1.0f;
            if (o < gc) {
                q = P.pos_s[gb + o];
                h = P.h ? P.h[P.perm[gb + o]] : P.h_const;
                bad = bad || !(h > 0.0f && h < INFINITY);
                bx0 = fminf(bx0, q.x); by0 = fminf(by0, q.y); bz0 = fminf(bz0, q.z);
                bx1 = fmaxf(bx1, q.x); by1 = fmaxf(by1, q.y); bz1 = fmaxf(bz1, q.z);
                hmax = fmaxf(hmax, h);
            }
            xi[t] = q.x; yi[t] = q.y; zi[t] = q.z;
            h2[t] = __fmul_rn(h, h);
            hinv[t] = 1.0f / h;
            cw[t] = 8.0f / (3.14159265358979f * h * h * h);
            cnt[t] = 0;
            rho[t] = 0.0f;
        }
        if (__any_sync(BH_FULL_MASK, bad)) {
            if (lane == 0) bh_set_error(ctrl, BH_ERR_NONFINITE);
            break;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bx0 = fminf(bx0, __shfl_xor_sync(BH_FULL_MASK, bx0, o));
            by0 = fminf(by0, __shfl_xor_sync(BH_FULL_MASK, by0, o));
            bz0 = fminf(bz0, __shfl_xor_sync(BH_FULL_MASK, bz0, o));
            bx1 = fmaxf(bx1, __shfl_xor_sync(BH_FULL_MASK, bx1, o));
            by1 = fmaxf(by1, __shfl_xor_sync(BH_FULL_MASK, by1, o));
            bz1 = fmaxf(bz1, __shfl_xor_sync(BH_FULL_MASK, bz1, o));
            hmax = fmaxf(hmax, __shfl_xor_sync(BH_FULL_MASK, hmax, o));
        }
        const float reach2 = hmax * hmax * (1.0f + 1e-5f);
#if BH_SPH_LEAF_FILTER
        // each target's own reach for the leaf filter (-1: no target in the slot)
        float reach_t[T];
#pragma unroll
        for (int t = 0; t < T; t++) reach_t[t] = (t * 32 + lane < gc) ? h2[t] * (1.0f + 1e-5f) : -1.0f;
#endif

        // root of the group's system
        int root = 0;
        for (int hi = n_roots; hi - root > 1;) {
            const int mid = (root + hi) >> 1;
            if (P.rec[mid].x <= gb) root = mid;
            else hi = mid;
        }
        int sp = 1, ring_head = 0, ring_cnt = 0;
        if (lane == 0) S.stack[0] = (uint32_t)root << 3;
        __syncwarp();
        bool overflow = false;
        while (sp > 0) {
            // pop the top 32 nodes
            int c = 0;
            uint32_t e = 0u;
            if (lane < sp) {
                e = S.stack[sp - 1 - lane];
                c = (int)(e & 7u) + 1;
            }
            const int incl = bh_warp_incl_scan(c);
            const int excl = incl - c;
            const int take = max(0, min(c, 32 - excl));
            const int st = (int)(e >> 3);
            for (int t = 0; t < take; t++) S.staging[excl + t] = (uint32_t)(st + t);
            const bool full = (lane < sp) && (take == c);
            const int nfull = __popc(__ballot_sync(BH_FULL_MASK, full));
            const int npop = min(__shfl_sync(BH_FULL_MASK, incl, 31), 32);
            __syncwarp();
            if (lane == nfull && lane < sp && take > 0)
                S.stack[sp - 1 - lane] = ((uint32_t)(st + take) << 3) | (uint32_t)(c - take - 1);
            sp -= nfull;
            const bool has = lane < npop;
            const int v = has ? (int)S.staging[lane] : 0;
            __syncwarp();

            // distance_test: the node's box against the group's box
            int4 r = make_int4(0, 0, -1, 0);
            bool near = false;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (has) {
                r = P.rec[v];
                a = P.blo[v];
                b = P.bhi[v];
                const float gx = fmaxf(fmaxf(a.x - bx1, bx0 - b.x), 0.0f);
                const float gy = fmaxf(fmaxf(a.y - by1, by0 - b.y), 0.0f);
                const float gz = fmaxf(fmaxf(a.z - bz1, bz0 - b.z), 0.0f);
                near = gx * gx + gy * gy + gz * gz <= reach2;
            }
            bool leaf = near && r.z < 0;
            const bool opn = near && r.z >= 0;
#if BH_SPH_LEAF_FILTER
            // per-target filter: a leaf near the group's box is kept only when
            // its box lies within reach of at least one target of the warp
            {
                unsigned int lm0 = __ballot_sync(BH_FULL_MASK, leaf), keep = 0u;
                while (lm0) {
                    const int q = __ffs(lm0) - 1;
                    lm0 &= lm0 - 1u;
                    const float lx0 = __shfl_sync(BH_FULL_MASK, a.x, q), ly0 = __shfl_sync(BH_FULL_MASK, a.y, q);
                    const float lz0 = __shfl_sync(BH_FULL_MASK, a.z, q), lx1 = __shfl_sync(BH_FULL_MASK, b.x, q);
                    const float ly1 = __shfl_sync(BH_FULL_MASK, b.y, q), lz1 = __shfl_sync(BH_FULL_MASK, b.z, q);
                    bool hit = false;
#pragma unroll
                    for (int t = 0; t < T; t++) {
                        const float dx = fmaxf(fmaxf(lx0 - xi[t], xi[t] - lx1), 0.0f);
                        const float dy = fmaxf(fmaxf(ly0 - yi[t], yi[t] - ly1), 0.0f);
                        const float dz = fmaxf(fmaxf(lz0 - zi[t], zi[t] - lz1), 0.0f);
                        hit = hit || (dx * dx + dy * dy + dz * dz <= reach_t[t]);
                    }
                    if (__any_sync(BH_FULL_MASK, hit)) keep |= 1u << q;
                }
                leaf = leaf && ((keep >> lane) & 1u);
            }
#endif
            const unsigned int om = __ballot_sync(BH_FULL_MASK, opn);
            if (sp + __popc(om) > kSphStackCap) {
                overflow = true;
                break;
            }
            if (opn) S.stack[sp + __popc(om & lt)] = ((uint32_t)r.z << 3) | (uint32_t)(r.w - 1);
            sp += __popc(om);

            // leaves: their particle ranges become candidates
            const unsigned int lm = __ballot_sync(BH_FULL_MASK, leaf);
            const int lq_n = __popc(lm);
            if (leaf) S.leafq[__popc(lm & lt)] = make_int2(r.x, r.y);
            __syncwarp();
            int lq_pos = 0;
            for (;;) {
                if (ring_cnt >= 32) {
                    bh_sph_tile<T>(S.ring + ring_head, S.ridx + ring_head, gb, xi, yi, zi, h2, hinv, cw, tn, cnt,
                                   rho);
                    tested += 32ull * (unsigned long long)gc;
                    ring_head ^= 32;
                    ring_cnt -= 32;
                    __syncwarp();
                    continue;
                }
                if (lq_pos >= lq_n) break;
                int c2 = 0;
                int2 q = make_int2(0, 0);
                if (lq_pos + lane < lq_n) {
                    q = S.leafq[lq_pos + lane];
                    c2 = q.y;
                }
                const int inc2 = bh_warp_incl_scan(c2);
                const int ex2 = inc2 - c2;
                const int take2 = max(0, min(c2, 32 - ex2));
                for (int t = 0; t < take2; t++) S.staging[ex2 + t] = (uint32_t)(q.x + t);
                const bool full2 = (lq_pos + lane < lq_n) && (take2 == c2);
                const int nf2 = __popc(__ballot_sync(BH_FULL_MASK, full2));
                const int nfill = min(__shfl_sync(BH_FULL_MASK, inc2, 31), 32);
                __syncwarp();
                if (lane == nf2 && lq_pos + lane < lq_n && take2 > 0)
                    S.leafq[lq_pos + lane] = make_int2(q.x + take2, c2 - take2);
                lq_pos += nf2;
                if (lane < nfill) {
                    const int k = (int)S.staging[lane];
                    const int slot = (ring_head + ring_cnt + lane) & (kSphRing - 1);
                    S.ring[slot] = P.pos_s[k];
                    S.ridx[slot] = k;
                }
                ring_cnt += nfill;
                __syncwarp();
            }
        }
        if (overflow) {
            if (lane == 0) bh_set_error(ctrl, BH_ERR_CAPACITY);
            break;
        }
        if (ring_cnt > 0) {
            // pad with far, massless candidates that match no index
            if (lane >= ring_cnt) {
                S.ring[ring_head + lane] = make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
                S.ridx[ring_head + lane] = -1;
            }
            __syncwarp();
            bh_sph_tile<T>(S.ring + ring_head, S.ridx + ring_head, gb, xi, yi, zi, h2, hinv, cw, tn, cnt, rho);
            tested += (unsigned long long)ring_cnt * (unsigned long long)gc;
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < T; t++) {
            const int o = t * 32 + lane;
            if (o < gc) {
                const uint32_t dst = P.perm[gb + o];
                if (P.count) P.count[dst] = cnt[t];
                if (P.rho) P.rho[dst] = rho[t];
            }
        }
    }
    if (lane == 0) {
        atomicAdd(&ctrl->n_pp, tested);
        atomicAdd(&ctrl->cum_pp, tested);
    }
}

__global__ void bh_sph_reset_kernel(bh_dev_ctrl* c)
{
    c->group_ctr = 0u;
    c->n_pp = 0ull;
    c->n_pc = 0ull;
}

// persistent grid: as many blocks per SM as the registers and shared memory allow
template <int T>
static int bh_sph_launch(const SphParams& P, int sm_count, cudaStream_t s)
{
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, bh_sph_kernel<T>, 128, 0) != cudaSuccess || bps < 1) {
        cudaGetLastError();
        bps = 4;
    }
    bh_sph_kernel<T><<<sm_count * bps, 128, 0, s>>>(P);
    return BH_OK;
}

int launch_sph(const float4* pos_s, const uint32_t* perm, const int32_t* g_first, const int32_t* g_count,
               const bh_nodes& nd, float4* blo, float4* bhi, int G, const float* h, float h_const, int32_t* count,
               float* rho, bh_dev_ctrl* ctrl, int sm_count, int grid, int max_level, cudaStream_t s)
{
    for (int lev = max_level; lev >= 0; lev--)
        bh_node_box_kernel<<<grid, 256, 0, s>>>(pos_s, nd.rec, blo, bhi, lev, ctrl);
    bh_sph_reset_kernel<<<1, 1, 0, s>>>(ctrl);
    SphParams P;
    P.pos_s = pos_s;
    P.perm = perm;
    P.g_first = g_first;
    P.g_count = g_count;
    P.rec = nd.rec;
    P.blo = blo;
    P.bhi = bhi;
    P.h = h;
    P.h_const = h_const;
    P.count = count;
    P.rho = rho;
    P.ctrl = ctrl;
    const int T = G <= 32 ? 1 : G <= 64 ? 2 : G <= 96 ? 3 : G <= 128 ? 4 : 8;
    switch (T) {
        case 1: return bh_sph_launch<1>(P, sm_count, s);
        case 2: return bh_sph_launch<2>(P, sm_count, s);
        case 3: return bh_sph_launch<3>(P, sm_count, s);
        case 4: return bh_sph_launch<4>(P, sm_count, s);
        default: return bh_sph_launch<8>(P, sm_count, s);
    }
}

}  // namespace bh

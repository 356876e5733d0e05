// bh_pwalk.cu -- the paper's own per-particle walk (Sec. 4.4, Fig. 5,
// Appendix A) on the device tree.
//
// Every node gets the two links of Fig. 5: "more" (its first child, the
// breadth-first child range's start) and "next" (the node that follows its
// subtree in depth-first order: the next sibling, else the parent's next).
// One thread walks the tree for one particle without a stack: an accepted
// cell (Eq. 2, d^2 > S_eff with d = |x_i - COM|, the node not holding i) or a
// rejected leaf is applied and the walk jumps to next; a rejected internal
// node continues at more.  A node holding a single particle is a
// particle-particle term.  Threads take particles in Morton order, so a warp
// walks nearby particles and its lanes follow similar paths.
//
// Accumulation: FP32 terms summed in runs of up to 32, each run added to the
// totals with Kahan compensation (as the group walk's tiles).  With
// BH_PWALK_UNSOFTENED_CELLS the particle-cell term uses eps = 0, as the
// Appendix A kernel does; particle-particle terms are always softened.
#include <algorithm>

#include "bh_internal.cuh"

namespace bh {

constexpr int kPWalkThreads = 128;
constexpr int kLinkDepthCap = 32;  // > the 22 levels of a 63-bit key tree

// parent of every node; roots (level 0, one per system) get -1
__global__ void bh_parent_kernel(const int4* __restrict__ rec, int32_t* __restrict__ parent,
                                 const bh_dev_ctrl* __restrict__ c)
{
    const int nn = (int)c->n_nodes, n_roots = (int)c->level_offset[1];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
        const int4 r = rec[v];
        if (v < n_roots) parent[v] = -1;
        for (int k = 0; k < r.w; k++) parent[r.z + k] = v;
    }
}

// next link: climb while the node is its parent's last child
__global__ void bh_next_kernel(const int4* __restrict__ rec, const int32_t* __restrict__ parent,
                               int32_t* __restrict__ next, bh_dev_ctrl* __restrict__ c)
{
    const int nn = (int)c->n_nodes;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
        int u = v, nx = -1, d = 0;
        for (; d < kLinkDepthCap; d++) {
            const int p = parent[u];
            if (p < 0) break;
            const int4 rp = rec[p];
            if (u < rp.z + rp.w - 1) {
                nx = u + 1;
                break;
            }
            u = p;
        }
        if (d == kLinkDepthCap) bh_set_error(c, BH_ERR_CAPACITY);
        next[v] = nx;
    }
}

struct PWalkParams {
    const float* soft_h;     // individual softening: eps_i^2 / 2 per particle (key order)
    const float* soft_hbar;  //   and the mass-weighted mean of it per node
    bool soft_cells;         //   cells softened (not BH_PWALK_UNSOFTENED_CELLS)
    const float4* pos_s;
    const uint32_t* perm;
    const int4* rec;
    const float4* com_m;
    const float* seff;
    const float4* quad;
    const int32_t* next;
    float4* out;
    bh_dev_ctrl* ctrl;
    int n;
    float eps2;   // particle-particle softening
    float eps2c;  // particle-cell softening (0 when unsoftened)
};

struct PSum {
    float x, y, z, p;        // current run
    float sx, sy, sz, sp;    // totals
    float cx, cy, cz, cp;    // Kahan compensations
    int k;                   // terms in the current run
};

__device__ __forceinline__ void bh_pk(float& s, float& c, float v)
{
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}
__device__ __forceinline__ void bh_pflush(PSum& S)
{
    bh_pk(S.sx, S.cx, S.x);
    bh_pk(S.sy, S.cy, S.y);
    bh_pk(S.sz, S.cz, S.z);
    bh_pk(S.sp, S.cp, S.p);
    S.x = S.y = S.z = S.p = 0.0f;
    S.k = 0;
}
__device__ __forceinline__ void bh_pcount(PSum& S)
{
    if (++S.k == 32) bh_pflush(S);
}

// particle-particle term of Eq. (1): a += m (x_j - x_i) / r^3, phi -= m / r
__device__ __forceinline__ void bh_p_pp(float4 s, float eps2, float xi, float yi, float zi, PSum& S)
{
    const float dx = s.x - xi, dy = s.y - yi, dz = s.z - zi;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
    const float ri = rsqrtf(r2);
    const float mr = s.w * ri;
    const float mr3 = mr * ri * ri;
    S.x = fmaf(mr3, dx, S.x);
    S.y = fmaf(mr3, dy, S.y);
    S.z = fmaf(mr3, dz, S.z);
    S.p -= mr;
    bh_pcount(S);
}

// particle-cell term: monopole, plus (ORDER 2) the second-order term of the
// softened kernel about the centre of mass.  With r = x_i - c, h^2 = r^2 +
// eps^2, g_n = h^-n, I the second moment (b = Ixx Iyy Izz Ixy, e = Ixz Iyz
// 1.5T 0.5T), q = r.I.r:
//   a += -M g3 r + 3 g5 I r + (1.5 T g5 - 7.5 q g7) r
//   phi += -M g1 - 1.5 q g5 + 0.5 T g3
template <int ORDER>
__device__ __forceinline__ void bh_p_pc(float4 c, const float4* __restrict__ q2, float eps2, float xi, float yi,
                                        float zi, PSum& S)
{
    const float rx = xi - c.x, ry = yi - c.y, rz = zi - c.z;
    const float h2 = fmaf(rz, rz, fmaf(ry, ry, fmaf(rx, rx, eps2)));
    const float g1 = rsqrtf(h2);
    const float g2 = g1 * g1;
    const float g3 = g1 * g2;
    float k = -c.w * g3, phi = -c.w * g1;
    float ax = 0.f, ay = 0.f, az = 0.f;
    if (ORDER >= 2) {
        const float4 b = q2[0], e = q2[1];
        const float g5 = g3 * g2, g7 = g5 * g2;
        const float u0 = fmaf(b.w, ry, fmaf(e.x, rz, b.x * rx));
        const float u1 = fmaf(b.w, rx, fmaf(e.y, rz, b.y * ry));
        const float u2 = fmaf(e.x, rx, fmaf(e.y, ry, b.z * rz));
        const float q = fmaf(rx, u0, fmaf(ry, u1, rz * u2));
        k = fmaf(e.z, g5, fmaf(-7.5f * q, g7, k));
        const float g5x3 = 3.0f * g5;
        ax = g5x3 * u0;
        ay = g5x3 * u1;
        az = g5x3 * u2;
        phi = fmaf(e.w, g3, fmaf(-1.5f * q, g5, phi));
    }
    S.x += fmaf(k, rx, ax);
    S.y += fmaf(k, ry, ay);
    S.z += fmaf(k, rz, az);
    S.p += phi;
    bh_pcount(S);
}

// IND: individual softening (symmetrized): a particle term softens with
// h_i + h_j, a cell term with h_i + hbar_c (h = eps^2 / 2), instead of eps^2.
template <int ORDER, bool IND>
__global__ void __launch_bounds__(kPWalkThreads) bh_pwalk_kernel(PWalkParams P)
{
    bh_dev_ctrl* ctrl = P.ctrl;
    const int n_roots = (int)ctrl->level_offset[1];
    unsigned long long cnt_pp = 0ull, cnt_pc = 0ull;
    const int stride = gridDim.x * blockDim.x;
    const int n_iter = (P.n + stride - 1) / stride;  // same trip count for every lane
    for (int it = 0; it < n_iter; it++) {
        const int i = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
        if (i < P.n) {
            const float4 xi = P.pos_s[i];
            const float hi = IND ? P.soft_h[i] : 0.0f;
            PSum S;
            S.x = S.y = S.z = S.p = S.sx = S.sy = S.sz = S.sp = S.cx = S.cy = S.cz = S.cp = 0.0f;
            S.k = 0;
            // the particle's root (one per system): the last level-0 node starting at or before i
            int v = 0;
            for (int hi = n_roots; hi - v > 1;) {
                const int mid = (v + hi) >> 1;
                if (P.rec[mid].x <= i) v = mid;
                else hi = mid;
            }
            const int root_next = P.next[v];
            while (v >= 0 && v != root_next) {
                const int4 r = P.rec[v];
                if (r.y == 1) {
                    if (r.x != i) {
                        bh_p_pp(P.pos_s[r.x], IND ? hi + P.soft_h[r.x] : P.eps2, xi.x, xi.y, xi.z, S);
                        cnt_pp++;
                    }
                    v = P.next[v];
                    continue;
                }
                const float4 c = P.com_m[v];
                const float dx = c.x - xi.x, dy = c.y - xi.y, dz = c.z - xi.z;
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                const bool holds = (r.x <= i) && (i < r.x + r.y);
                if (d2 > P.seff[v] && !holds) {
                    const float e2c = IND ? (P.soft_cells ? hi + P.soft_hbar[v] : 0.0f) : P.eps2c;
                    bh_p_pc<ORDER>(c, ORDER >= 2 ? P.quad + 2 * (size_t)v : nullptr, e2c, xi.x, xi.y, xi.z, S);
                    cnt_pc++;
                    v = P.next[v];
                } else if (r.z < 0) {
                    for (int j = r.x; j < r.x + r.y; j++) {
                        if (j == i) continue;
                        bh_p_pp(P.pos_s[j], IND ? hi + P.soft_h[j] : P.eps2, xi.x, xi.y, xi.z, S);
                    }
                    cnt_pp += (unsigned long long)(r.y - (holds ? 1 : 0));
                    v = P.next[v];
                } else {
                    v = r.z;
                }
            }
            bh_pflush(S);
            P.out[P.perm[i]] = make_float4(S.sx - S.cx, S.sy - S.cy, S.sz - S.cz, S.sp - S.cp);
        }
    }
    // interaction counters: one atomic per warp
    for (int o = 16; o > 0; o >>= 1) {
        cnt_pp += __shfl_down_sync(BH_FULL_MASK, cnt_pp, o);
        cnt_pc += __shfl_down_sync(BH_FULL_MASK, cnt_pc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ctrl->n_pp, cnt_pp);
        atomicAdd(&ctrl->n_pc, cnt_pc);
        atomicAdd(&ctrl->cum_pp, cnt_pp);
        atomicAdd(&ctrl->cum_pc, cnt_pc);
    }
}

__global__ void bh_pwalk_reset_kernel(bh_dev_ctrl* c)
{
    c->n_pp = 0ull;
    c->n_pc = 0ull;
}

// Individual softening, step 1: h = eps^2 / 2 of every particle in key order
// (a negative or non-finite length is reported as BH_ERR_NONFINITE).
__global__ void __launch_bounds__(256) bh_soft_gather_kernel(const float* __restrict__ eps,
                                                             const uint32_t* __restrict__ perm, int n,
                                                             float* __restrict__ h, bh_dev_ctrl* c)
{
    bool bad = false;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const float e = eps[perm[k]];
        bad |= !(e >= 0.0f && isfinite(e));
        h[k] = 0.5f * (e * e);
    }
    if (__any_sync(BH_FULL_MASK, bad) && (threadIdx.x & 31) == 0) atomicCAS(&c->status, 0u, (unsigned int)(-BH_ERR_NONFINITE));
}

// Step 2, one level (deepest first): per node the FP64 sums (sum m, sum m h)
// over its particles (leaves) or its children, and hbar = sum m h / sum m.
__global__ void __launch_bounds__(256) bh_soft_level_kernel(const float4* __restrict__ pos_s,
                                                            const float* __restrict__ h, bh_nodes nd, int lev,
                                                            double2* __restrict__ sums, float* __restrict__ hbar,
                                                            const bh_dev_ctrl* __restrict__ c)
{
    if (c->n_nodes == 0u) return;
    const int v0 = (int)c->level_offset[lev], v1 = (int)c->level_offset[lev + 1];
    for (int v = v0 + blockIdx.x * blockDim.x + threadIdx.x; v < v1; v += gridDim.x * blockDim.x) {
        const int4 r = nd.rec[v];
        double sm = 0.0, se = 0.0;
        if (r.z < 0) {
            for (int j = r.x; j < r.x + r.y; j++) {
                const double m = pos_s[j].w;
                sm += m;
                se += m * (double)h[j];
            }
        } else {
            for (int k = 0; k < r.w; k++) {
                const double2 t = sums[r.z + k];
                sm += t.x;
                se += t.y;
            }
        }
        sums[v] = make_double2(sm, se);
        hbar[v] = sm != 0.0 ? (float)(se / sm) : 0.0f;
    }
}

void launch_softening(const float* eps, const uint32_t* perm, const float4* pos_s, const bh_nodes& nd, int n,
                      bool deep, const bh_soft& soft, bh_dev_ctrl* ctrl, int grid, cudaStream_t s)
{
    bh_soft_gather_kernel<<<grid, 256, 0, s>>>(eps, perm, n, soft.h, ctrl);
    for (int lev = deep ? BH_MAX_LEVEL_DEEP : BH_MAX_LEVEL; lev >= 0; lev--)
        bh_soft_level_kernel<<<grid, 256, 0, s>>>(pos_s, soft.h, nd, lev, soft.sums, soft.hbar, ctrl);
}

int launch_pwalk(const float4* pos_s, const uint32_t* perm, const bh_nodes& nd, int32_t* parent, int32_t* next,
                 int order, int n, int node_cap, float eps, bool unsoftened_cells, float4* out, bh_dev_ctrl* ctrl,
                 int sm_count, cudaStream_t s, const bh_soft* soft)
{
    const int link_grid = std::max(1, std::min((node_cap + 255) / 256, sm_count * 16));
    bh_parent_kernel<<<link_grid, 256, 0, s>>>(nd.rec, parent, ctrl);
    bh_next_kernel<<<link_grid, 256, 0, s>>>(nd.rec, parent, next, ctrl);
    bh_pwalk_reset_kernel<<<1, 1, 0, s>>>(ctrl);
    PWalkParams P;
    P.pos_s = pos_s;
    P.perm = perm;
    P.rec = nd.rec;
    P.com_m = nd.com_m;
    P.seff = nd.seff;
    P.quad = nd.quad;
    P.next = next;
    P.out = out;
    P.ctrl = ctrl;
    P.n = n;
    P.eps2 = eps * eps;
    P.eps2c = unsoftened_cells ? 0.0f : eps * eps;
    P.soft_h = soft ? soft->h : nullptr;
    P.soft_hbar = soft ? soft->hbar : nullptr;
    P.soft_cells = !unsoftened_cells;
    const int grid = std::max(1, std::min((n + kPWalkThreads - 1) / kPWalkThreads, sm_count * 64));
    if (soft) {
        if (order >= 2) bh_pwalk_kernel<2, true><<<grid, kPWalkThreads, 0, s>>>(P);
        else bh_pwalk_kernel<1, true><<<grid, kPWalkThreads, 0, s>>>(P);
    } else {
        if (order >= 2) bh_pwalk_kernel<2, false><<<grid, kPWalkThreads, 0, s>>>(P);
        else bh_pwalk_kernel<1, false><<<grid, kPWalkThreads, 0, s>>>(P);
    }
    return BH_OK;
}

}  // namespace bh

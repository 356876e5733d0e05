// bh_walk.cu -- group tree walk and force evaluation (step 5 of the paper's
// flow, Sec. 4.4; Fig. 3 / Fig. 5 walk, Eq. 1 interactions, Eq. 2 criterion).
//
// The paper walks the tree once per particle with the next/more pointers of
// Fig. 5 (bh_pwalk.cu has that form).  Here one warp walks the tree once for
// a whole group of up to 32*T key-contiguous particles (the GRAPE-style
// shared interaction list of Sec. 4.2, built on the device): nodes are tested
// 32 at a time, one per lane, against the group's bounding box.  A node is
// accepted when the squared distance from its centre of mass to the box
// exceeds S_eff (Eq. 2 made conservative for every member) and it holds no
// group member; accepted nodes become particle-cell sources, rejected leaves
// contribute their particles as particle-particle sources, other rejected
// nodes are opened.
// Sources go through a 128-entry ring in shared memory and are evaluated in
// tiles of 64: every lane applies each source to its T targets in FP32 with
// rsqrtf, two sources per packed f32x2 instruction; each tile's partial sums
// (plain FP32 sums of 32 terms per pair half) are added to the running totals
// with Kahan compensation.  A target slot
// holding few targets is split across source phases (see Layout).  The
// group's own particles are applied once, as a masked "self" tile, so the
// target itself is excluded by index.
//
// Stack bound: entries are ranges of <= 8 sibling nodes.  A pop takes the top
// 32 nodes; all entries above the deepest one touched are consumed, so after
// a pop the stack holds only levels below those popped, and the pushes of one
// pop (<= 32 ranges) are the only entries of their levels.  Hence at most 33
// ranges per level 1..21 are ever stored (21 = the deepest level of 63-bit
// keys): kStackCap = 704 cannot overflow (overflow is still checked and
// reported as BH_ERR_CAPACITY).
#include "bh_mlp.cuh"

namespace bh {

constexpr int kStackCap = 704;
constexpr int kTile = 64;              // sources per tile (one Kahan-compensated addition per tile)
constexpr int kTilePairs = kTile / 2;  // a tile as even/odd source pairs
constexpr int kRing = 2 * kTile;       // sources per ring (two tiles), stored as even/odd pairs
// unroll factors of the per-tile pair loops (tuning constants, measured:
// larger factors overflow the instruction cache, as every T-slot variant of
// the loops is live at once across the SM's warps)
#ifndef BH_POINT_UNROLL
#define BH_POINT_UNROLL 4
#endif
#ifndef BH_POINT_UNROLL_LEARNED
#define BH_POINT_UNROLL_LEARNED 4
#endif
#ifndef BH_QUAD_UNROLL
#define BH_QUAD_UNROLL 2           // one-warp kernel (the paired and TMA kernels keep 1)
#endif
#ifndef BH_QUAD_UNROLL_LEARNED
#define BH_QUAD_UNROLL_LEARNED 1    // the learned walk (more registers for the network)
#endif
constexpr int kPointUnroll = BH_POINT_UNROLL;
constexpr int kPointUnrollLearned = BH_POINT_UNROLL_LEARNED;
constexpr int kPointUnrollPaired = 2;
constexpr int kQuadUnroll = BH_QUAD_UNROLL;
constexpr int kQuadUnrollLearned = BH_QUAD_UNROLL_LEARNED;
constexpr int kQuadUnrollPaired = 1;
constexpr int kQuadUnrollTma = 1;

// Quadrupole-pair unroll of the one-warp kernel: 2 up to 3 slots per lane;
// the 4-slot and learned kernels, with more registers live, keep 1.
template <int T, bool LEARNED>
__host__ __device__ constexpr int bh_quad_unroll() { return LEARNED ? kQuadUnrollLearned : (T <= 3 ? kQuadUnroll : 1); }

// Sources are staged negated and as pairs (ring positions 2p, 2p+1 side by
// side) so that the interaction arithmetic runs on packed f32x2 operations:
// one instruction computes the same step for two sources.
struct WarpSmem {
    float gbox[8];              // the group's box: xmin, ymin, zmin, radius, xmax, ymax, zmax, -
    unsigned long long tot[2];  // interactions so far: particle-particle, particle-cell
    uint32_t stack[kStackCap];  // (first node << 3) | (count - 1)
    uint32_t staging[32];
    int2 leafq[64];             // pending particle ranges (first, count)
    float4 ra[kRing / 2];       // point sources: (-x, -x', -y, -y')
    float4 rb[kRing / 2];       //                (-z, -z', -m, -m')
};
struct WarpQuad {               // quadrupole cells, pairs as above; Q = 3 I - T 1 (traceless), T = tr I
    float4 a[kRing / 2];        // (-x, -x', -y, -y')      centre of mass
    float4 b[kRing / 2];        // (-z, -z', -M, -M')
    float4 c[kRing / 2];        // (Qxx, Qxx', Qyy, Qyy')
    float4 d[kRing / 2];        // (Qzz, Qzz', Qxy, Qxy')
    float4 e[kRing / 2];        // (Qxz, Qxz', Qyz, Qyz')
    float4 f[kRing / 2];        // (-T eps^2, -T' eps^2, -, -)
};

__device__ __forceinline__ void bh_put_point(WarpSmem& S, int r, float4 v)
{
    float* a = reinterpret_cast<float*>(&S.ra[r >> 1]) + (r & 1);
    float* b = reinterpret_cast<float*>(&S.rb[r >> 1]) + (r & 1);
    a[0] = -v.x; a[2] = -v.y;
    b[0] = -v.z; b[2] = -v.w;
}
// cell with centre/mass cm and stored moments qb = (Ixx, Iyy, Izz, Ixy),
// qc = (Ixz, Iyz, 1.5 T, 0.5 T): staged as the traceless Q = 3 I - T 1 and
// -T eps^2 (see bh_pq2)
__device__ __forceinline__ void bh_put_quad(WarpQuad& Q, int r, float4 cm, float4 qb, float4 qc, float eps2)
{
    const int p = r >> 1, h = r & 1;
    float* a = reinterpret_cast<float*>(&Q.a[p]) + h;
    float* b = reinterpret_cast<float*>(&Q.b[p]) + h;
    float* c = reinterpret_cast<float*>(&Q.c[p]) + h;
    float* d = reinterpret_cast<float*>(&Q.d[p]) + h;
    float* e = reinterpret_cast<float*>(&Q.e[p]) + h;
    float* f = reinterpret_cast<float*>(&Q.f[p]) + h;
    const float T = 2.0f * qc.w;  // exact
    a[0] = -cm.x; a[2] = -cm.y;
    b[0] = -cm.z; b[2] = -cm.w;
    c[0] = __fmaf_rn(3.0f, qb.x, -T); c[2] = __fmaf_rn(3.0f, qb.y, -T);
    d[0] = __fmaf_rn(3.0f, qb.z, -T); d[2] = 3.0f * qb.w;
    e[0] = 3.0f * qc.x; e[2] = 3.0f * qc.y;
    f[0] = -T * eps2;
}

struct WalkParams {
    const float4* pos_s;
    const uint32_t* perm;
    const int32_t* g_first;
    const int32_t* g_count;
    const int4* rec;
    const float4* com_m;
    const float* seff;
    const float4* quad;
    float4* out;
    bh_dev_ctrl* ctrl;
    float eps2;
    // learned criterion
    const float4* mfeat;     // node-constant features
    const bh_mlp_dev* mlp;   // network (global copy)
    float theta_guard;       // theta of the S_eff in use (the guard)
    const float4* wrec;      // walk records (TMA-staged walk)
};

// Running totals of a lane's T targets with their Kahan compensations, the
// latter either in registers or in shared memory (this lane's column of a
// per-warp [4T][32] array: touched once per tile, they need no register).
#ifndef BH_KAHAN_SMEM
#define BH_KAHAN_SMEM 1
#endif
template <int T>
struct Acc {
    float x[T], y[T], z[T], p[T];
#if BH_KAHAN_SMEM
    float* kc;
    __device__ __forceinline__ float& c(int t, int k) { return kc[(4 * t + k) * 32]; }
#else
    float cc[4][T];
    __device__ __forceinline__ float& c(int t, int k) { return cc[k][t]; }
#endif
};
template <int T>
__host__ __device__ constexpr size_t bh_kahan_smem_bytes()
{
    return BH_KAHAN_SMEM ? (size_t)T * 4 * 32 * sizeof(float) : 0;
}

// Squared distance of a node's centre of mass from the group's box, as
// explicit round-to-nearest operations: every walk kernel takes the same
// opening decisions bit for bit (an expression left to the compiler may be
// contracted into FMAs differently in each kernel, which flips near ties).
__device__ __forceinline__ float bh_dist2(float dx, float dy, float dz)
{
    return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Target layout of a group of gc particles on the warp's T slots per lane
// (warp-uniform).  Slots 0..nf-1 hold targets t*32 + lane.  When the last
// slot would hold at most kSplitMax targets (k = gc - 32*nf) it is "split":
// lane l holds target nf*32 + (l mod m), m = 2^lg >= k, and evaluates only
// the 2m sources of each tile in its phase (l / m); the phases' partial sums
// are added across lanes once, when the group ends.  A slot with 4 targets
// then costs 8 evaluations per tile instead of 64.
#ifndef BH_SPLIT_MAX
#define BH_SPLIT_MAX 16
#endif
constexpr int kSplitMax = BH_SPLIT_MAX;
struct Layout {
    int nf;      // full slots
    bool split;  // slot nf is split
    int lg;      // log2 of the targets per phase in the split slot
};

__device__ __forceinline__ void bh_kahan(float& s, float& c, float v)
{
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

typedef float2 f2;
__device__ __forceinline__ f2 bh_add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 bh_mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 bh_fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 bh_rsqrt2(f2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ f2 bh_lo(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ f2 bh_hi(float4 v) { return make_float2(v.z, v.w); }

// Per-slot partial sums of one tile, two lanes of a pair each.
template <int T>
struct Part {
    f2 x[T], y[T], z[T], p[T], q[T];
};

// Adds the tile's pair sums of slots 0..TN-1 to the running totals.
template <int T, int TN>
__device__ __forceinline__ void bh_add_tile(Acc<T>& A, const Part<T>& P, bool with_q)
{
#pragma unroll
    for (int t = 0; t < TN; t++) {
        float pt = P.p[t].x + P.p[t].y;
        if (with_q) pt = fmaf(-0.5f, P.q[t].x + P.q[t].y, pt);
        bh_kahan(A.x[t], A.c(t, 0), P.x[t].x + P.x[t].y);
        bh_kahan(A.y[t], A.c(t, 1), P.y[t].x + P.y[t].y);
        bh_kahan(A.z[t], A.c(t, 2), P.z[t].x + P.z[t].y);
        bh_kahan(A.p[t], A.c(t, 3), pt);
    }
}

// A pair of point sources (negated, as staged) on one target held twice in
// (x, y, z); Eq. 1:  a += m (s - x_i) / r^3,  phi -= m / r.
__device__ __forceinline__ void bh_pp2(float4 sa, float4 sb, f2 eps2, f2 x, f2 y, f2 z, f2& ax, f2& ay, f2& az,
                                       f2& ap)
{
    const f2 dx = bh_add2(x, bh_lo(sa)), dy = bh_add2(y, bh_hi(sa)), dz = bh_add2(z, bh_lo(sb));  // x_i - s
    const f2 r2 = bh_fma2(dz, dz, bh_fma2(dy, dy, bh_fma2(dx, dx, eps2)));
    const f2 ri = bh_rsqrt2(r2);
    const f2 mr = bh_mul2(bh_hi(sb), ri);          // -m / r
    const f2 mr3 = bh_mul2(mr, bh_mul2(ri, ri));   // -m / r^3
    ax = bh_fma2(mr3, dx, ax);
    ay = bh_fma2(mr3, dy, ay);
    az = bh_fma2(mr3, dz, az);
    ap = bh_add2(ap, mr);
}

// A pair of quadrupole cells on one target.  With r = x_i - c, h^2 = r^2 +
// eps^2, g_n = h^-n, the traceless Q = 3 I - T 1, u = Q r and
// s = r.u - T eps^2, the second-order term of the softened kernel is
//   a   += g5 u + k r,   k = -M g3 - 2.5 g5 g2 s
//   phi += -M g1 - 0.5 s g5
// (the same as  a += 3 g5 I r + (1.5 T g5 - 7.5 q g7) r,
// phi -= 0.5 (3 q g5 - T g3) with q = r.I.r, since 3 q = r.Q.r + T r^2 and
// r^2 = h^2 - eps^2); the last term accumulated apart (aq) and scaled once
// per tile.  33 FP32 operations per source (21 FMA, 9 mul, 3 add).
__device__ __forceinline__ void bh_pq2(float4 ca, float4 cb, float4 cc, float4 cd, float4 ce, float4 cf, f2 eps2,
                                       f2 x, f2 y, f2 z, f2& ax, f2& ay, f2& az, f2& ap, f2& aq)
{
    const f2 rx = bh_add2(x, bh_lo(ca)), ry = bh_add2(y, bh_hi(ca)), rz = bh_add2(z, bh_lo(cb));
    const f2 h2 = bh_fma2(rz, rz, bh_fma2(ry, ry, bh_fma2(rx, rx, eps2)));
    const f2 g1 = bh_rsqrt2(h2);
    const f2 g2 = bh_mul2(g1, g1);
    const f2 g3 = bh_mul2(g1, g2);
    const f2 g5 = bh_mul2(g3, g2);
    const f2 mneg = bh_hi(cb);
    const f2 u0 = bh_fma2(bh_hi(cd), ry, bh_fma2(bh_lo(ce), rz, bh_mul2(bh_lo(cc), rx)));
    const f2 u1 = bh_fma2(bh_hi(cd), rx, bh_fma2(bh_hi(ce), rz, bh_mul2(bh_hi(cc), ry)));
    const f2 u2 = bh_fma2(bh_lo(ce), rx, bh_fma2(bh_hi(ce), ry, bh_mul2(bh_lo(cd), rz)));
    const f2 sq = bh_fma2(rx, u0, bh_fma2(ry, u1, bh_fma2(rz, u2, bh_lo(cf))));
    const f2 w = bh_mul2(bh_mul2(sq, make_float2(-2.5f, -2.5f)), g2);
    const f2 k = bh_fma2(g5, w, bh_mul2(mneg, g3));
    ax = bh_fma2(g5, u0, bh_fma2(k, rx, ax));
    ay = bh_fma2(g5, u1, bh_fma2(k, ry, ay));
    az = bh_fma2(g5, u2, bh_fma2(k, rz, az));
    ap = bh_fma2(mneg, g1, ap);
    aq = bh_fma2(sq, g5, aq);
}

// Targets of a lane: slot t holds (x, x), (y, y), (z, z).
template <int T>
struct Tgt {
    f2 x[T], y[T], z[T];
};

// One tile (np <= kTilePairs pairs) of point sources on the first NF slots of every lane,
// the pair loop unrolled PU times.
template <int T, int NF, int PU>
__device__ __forceinline__ void bh_eval_points(const float4* __restrict__ ra, const float4* __restrict__ rb,
                                               f2 eps2, const Tgt<T>& X, Acc<T>& A, int np)
{
    Part<T> P;
#pragma unroll
    for (int t = 0; t < NF; t++) P.x[t] = P.y[t] = P.z[t] = P.p[t] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int j0 = 0; j0 < np; j0 += PU) {
#pragma unroll
        for (int j = j0; j < j0 + PU; j++) {
            const float4 sa = ra[j], sb = rb[j];
#pragma unroll
            for (int t = 0; t < NF; t++)
                bh_pp2(sa, sb, eps2, X.x[t], X.y[t], X.z[t], P.x[t], P.y[t], P.z[t], P.p[t]);
        }
    }
    bh_add_tile<T, NF>(A, P, false);
}

// One tile (np <= kTilePairs pairs) of quadrupole cells on the first NF slots of every lane.
// QC: any staging with the six pair arrays a..f of WarpQuad (pairs p0..p0+15).
template <int T, int NF, class QC, int QU>
__device__ __forceinline__ void bh_eval_quads(const QC& Q, int p0, f2 eps2, const Tgt<T>& X, Acc<T>& A, int np)
{
    Part<T> P;
#pragma unroll
    for (int t = 0; t < NF; t++) P.x[t] = P.y[t] = P.z[t] = P.p[t] = P.q[t] = make_float2(0.f, 0.f);
#pragma unroll QU
    for (int j = p0; j < p0 + np; j++) {
        const float4 ca = Q.a[j], cb = Q.b[j], cc = Q.c[j], cd = Q.d[j], ce = Q.e[j], cf = Q.f[j];
#pragma unroll
        for (int t = 0; t < NF; t++)
            bh_pq2(ca, cb, cc, cd, ce, cf, eps2, X.x[t], X.y[t], X.z[t], P.x[t], P.y[t], P.z[t], P.p[t], P.q[t]);
    }
    bh_add_tile<T, NF>(A, P, true);
}

// The split slot: its target, and the m = 2^lg sources of the lane's phase
// (pairs from p; with m = 1 the pair holding the lane's source, one half kept).
template <int T>
__device__ __forceinline__ void bh_split_target(const Layout& L, const Tgt<T>& X, f2& x, f2& y, f2& z)
{
    x = X.x[0]; y = X.y[0]; z = X.z[0];
#pragma unroll
    for (int t = 1; t < T; t++)
        if (t == L.nf) { x = X.x[t]; y = X.y[t]; z = X.z[t]; }
}
// With kTilePairs = 32 pairs per tile and 32 / m phases, a phase (and each
// of its lanes) takes m whole pairs: pairs (l / m) * m .. + m - 1.
static_assert(kTilePairs == 32, "split phases assume 32 pairs per tile");
__device__ __forceinline__ float bh_split_sum(const Layout&, f2 v) { return v.x + v.y; }
template <int T>
__device__ __forceinline__ void bh_split_add(const Layout& L, Acc<T>& A, float ax, float ay, float az, float ap)
{
#pragma unroll
    for (int t = 0; t < T; t++)
        if (t == L.nf) {
            bh_kahan(A.x[t], A.c(t, 0), ax);
            bh_kahan(A.y[t], A.c(t, 1), ay);
            bh_kahan(A.z[t], A.c(t, 2), az);
            bh_kahan(A.p[t], A.c(t, 3), ap);
        }
}
template <int T>
__device__ __forceinline__ void bh_split_points(const Layout& L, const float4* __restrict__ ra,
                                                const float4* __restrict__ rb, f2 eps2, const Tgt<T>& X, Acc<T>& A)
{
    f2 x, y, z, ax = make_float2(0.f, 0.f), ay = ax, az = ax, ap = ax;
    bh_split_target<T>(L, X, x, y, z);
    const int p = ((threadIdx.x & 31) >> L.lg) << L.lg, np = 1 << L.lg;
    for (int i = p; i < p + np; i++) bh_pp2(ra[i], rb[i], eps2, x, y, z, ax, ay, az, ap);
    bh_split_add<T>(L, A, bh_split_sum(L, ax), bh_split_sum(L, ay), bh_split_sum(L, az), bh_split_sum(L, ap));
}
template <int T, class QC>
__device__ __forceinline__ void bh_split_quads(const Layout& L, const QC& Q, int p0, f2 eps2, const Tgt<T>& X,
                                               Acc<T>& A)
{
    f2 x, y, z, ax = make_float2(0.f, 0.f), ay = ax, az = ax, ap = ax, aq = ax;
    bh_split_target<T>(L, X, x, y, z);
    const int p = p0 + (((threadIdx.x & 31) >> L.lg) << L.lg), np = 1 << L.lg;
    for (int i = p; i < p + np; i++)
        bh_pq2(Q.a[i], Q.b[i], Q.c[i], Q.d[i], Q.e[i], Q.f[i], eps2, x, y, z, ax, ay, az, ap, aq);
    bh_split_add<T>(L, A, bh_split_sum(L, ax), bh_split_sum(L, ay), bh_split_sum(L, az),
                    fmaf(-0.5f, bh_split_sum(L, aq), bh_split_sum(L, ap)));
}

// Dispatch on the warp-uniform layout.  Every bh_eval_* instance is reached
// from one call site only (they are inlined: a second site would double the
// code of the hottest loop).
template <int T, int PU = kPointUnroll>
// A point tile; np: pairs evaluated on the full slots (kTilePairs, or fewer
// for a group's last, partly padded tile: the padding pairs add exact zeros),
// a multiple of PU.  The split slot always takes the whole tile.
__device__ __forceinline__ void bh_points(const Layout& L, const float4* __restrict__ ra,
                                          const float4* __restrict__ rb, f2 eps2, const Tgt<T>& X, Acc<T>& A,
                                          int np = kTilePairs)
{
    if (T > 1 && L.nf == 1) bh_eval_points<T, 1, PU>(ra, rb, eps2, X, A, np);
    else if (T > 2 && L.nf == 2) bh_eval_points<T, (T > 2 ? 2 : T), PU>(ra, rb, eps2, X, A, np);
    else if (T > 3 && L.nf == 3) bh_eval_points<T, (T > 3 ? 3 : T), PU>(ra, rb, eps2, X, A, np);
    else if (T > 4 && L.nf == 4) bh_eval_points<T, (T > 4 ? 4 : T), PU>(ra, rb, eps2, X, A, np);
    else if (L.nf > 0) bh_eval_points<T, T, PU>(ra, rb, eps2, X, A, np);
    if (L.split) bh_split_points<T>(L, ra, rb, eps2, X, A);
}
// A quadrupole tile (pairs p0 ..); np as for bh_points (any count); QU: the
// unroll factor of the pair loop.
template <int T, class QC, int QU = kQuadUnroll>
__device__ __forceinline__ void bh_quads(const Layout& L, const QC& Q, int p0, f2 eps2, const Tgt<T>& X,
                                         Acc<T>& A, int np = kTilePairs)
{
    if (T > 1 && L.nf == 1) bh_eval_quads<T, 1, QC, QU>(Q, p0, eps2, X, A, np);
    else if (T > 2 && L.nf == 2) bh_eval_quads<T, (T > 2 ? 2 : T), QC, QU>(Q, p0, eps2, X, A, np);
    else if (T > 3 && L.nf == 3) bh_eval_quads<T, (T > 3 ? 3 : T), QC, QU>(Q, p0, eps2, X, A, np);
    else if (T > 4 && L.nf == 4) bh_eval_quads<T, (T > 4 ? 4 : T), QC, QU>(Q, p0, eps2, X, A, np);
    else if (L.nf > 0) bh_eval_quads<T, T, QC, QU>(Q, p0, eps2, X, A, np);
    if (L.split) bh_split_quads<T, QC>(L, Q, p0, eps2, X, A);
}

// The group's own particles on its members, target itself masked.
// With a split slot, only its phase-0 lanes (lane < m) keep their sums: the
// other phases hold copies of the same targets.
template <int T>
__device__ __forceinline__ void bh_eval_self(int gc, const Layout& L, float eps2, const float (&xi)[T],
                                             const float (&yi)[T], const float (&zi)[T], const float (&mi)[T],
                                             Acc<T>& A)
{
    const int lane = threadIdx.x & 31;
    float tx[T], ty[T], tz[T], tp[T];
#pragma unroll
    for (int t = 0; t < T; t++) tx[t] = ty[t] = tz[t] = tp[t] = 0.0f;
#pragma unroll
    for (int t2 = 0; t2 < T; t2++) {
        for (int j = 0; j < 32; j++) {
            if (t2 * 32 + j >= gc) break;
            const float sx = __shfl_sync(BH_FULL_MASK, xi[t2], j);
            const float sy = __shfl_sync(BH_FULL_MASK, yi[t2], j);
            const float sz = __shfl_sync(BH_FULL_MASK, zi[t2], j);
            const float sm = __shfl_sync(BH_FULL_MASK, mi[t2], j);
#pragma unroll
            for (int t = 0; t < T; t++) {
                const bool self = (t == t2) && (lane == j);
                const float dx = sx - xi[t], dy = sy - yi[t], dz = sz - zi[t];
                float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
                r2 = self ? 1.0f : r2;
                const float ri = rsqrtf(r2);
                const float mr = __fmul_rn(self ? 0.0f : sm, ri);
                const float mr3 = __fmul_rn(__fmul_rn(mr, ri), ri);
                tx[t] = fmaf(mr3, dx, tx[t]);
                ty[t] = fmaf(mr3, dy, ty[t]);
                tz[t] = fmaf(mr3, dz, tz[t]);
                tp[t] = __fsub_rn(tp[t], mr);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < T; t++)
        if (L.split && t == L.nf && (lane >> L.lg) != 0) tx[t] = ty[t] = tz[t] = tp[t] = 0.0f;
#pragma unroll
    for (int t = 0; t < T; t++) {
        bh_kahan(A.x[t], A.c(t, 0), tx[t]);
        bh_kahan(A.y[t], A.c(t, 1), ty[t]);
        bh_kahan(A.z[t], A.c(t, 2), tz[t]);
        bh_kahan(A.p[t], A.c(t, 3), tp[t]);
    }
}

__device__ __forceinline__ float4 bh_pad_source() { return make_float4(1e18f, 1e18f, 1e18f, 0.0f); }

// The group box is read from shared memory at every batch of node tests
// rather than held in six registers across the walk: the tile loops of the
// three-slot kernel are at the register limit.  The load is explicit so that
// the compiler does not hoist it back into registers.
__device__ __forceinline__ float4 bh_lds4(const float* p)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(static_cast<unsigned int>(__cvta_generic_to_shared(p))));
    return v;
}

// resident blocks of 128 threads per SM (register budget 65536 / (128 * b))
#ifndef BH_WALK_MINB3
#define BH_WALK_MINB3 4
#endif
template <int T, bool LEARNED>
constexpr int bh_walk_min_blocks()
{
    return LEARNED ? (T <= 4 ? 3 : 2) : (T <= 1 ? 6 : T <= 2 ? 4 : T <= 3 ? BH_WALK_MINB3 : T <= 4 ? 3 : 2);
}

template <int T, int ORDER, bool LEARNED>
__global__ void __launch_bounds__(128, bh_walk_min_blocks<T, LEARNED>())
    bh_walk_kernel(WalkParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    WarpSmem& S = reinterpret_cast<WarpSmem*>(smem_raw)[wib];
    WarpQuad* Q = nullptr;
    if (ORDER >= 2) Q = reinterpret_cast<WarpQuad*>(smem_raw + (size_t)nwarps * sizeof(WarpSmem)) + wib;
    // learned criterion: the network (per block) and a feature staging area (per warp)
    unsigned char* lbase = smem_raw + (size_t)nwarps * (sizeof(WarpSmem) + (ORDER >= 2 ? sizeof(WarpQuad) : 0));
    bh_mlp_dev* MW = reinterpret_cast<bh_mlp_dev*>(lbase);
    uint32_t* xs = reinterpret_cast<uint32_t*>(lbase + sizeof(bh_mlp_dev)) + wib * (32 * 8);
    // Kahan compensations (per warp, after the learned-criterion area)
    unsigned char* kbase = lbase + (LEARNED ? sizeof(bh_mlp_dev) + (size_t)nwarps * 32 * 8 * sizeof(uint32_t) : 0);
    float* kcol = reinterpret_cast<float*>(kbase + (size_t)wib * bh_kahan_smem_bytes<T>()) + lane;
    if (LEARNED) {
        for (int i = threadIdx.x; i < (int)(sizeof(bh_mlp_dev) / 4); i += blockDim.x)
            reinterpret_cast<uint32_t*>(MW)[i] = reinterpret_cast<const uint32_t*>(P.mlp)[i];
        __syncthreads();
    }
    const unsigned int lt = bh_lanemask_lt();
    const float eps2 = P.eps2;
    bh_dev_ctrl* ctrl = P.ctrl;
    const int ng = (int)ctrl->n_groups;
    const int n_roots = (int)ctrl->level_offset[1];
    const float boxL = LEARNED ? ctrl->box[3] : 1.0f;
    if (lane == 0) S.tot[0] = S.tot[1] = 0ull;

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&ctrl->group_ctr, 1u);
        g = __shfl_sync(BH_FULL_MASK, g, 0);
        if (g >= ng) break;
        int ab = 0;
        if (lane == 0) ab = (int)*(volatile unsigned int*)&ctrl->abort;
        if (__shfl_sync(BH_FULL_MASK, ab, 0)) break;
        const int gb = P.g_first[g], gc = P.g_count[g], ge = gb + gc;
        const int tn = (gc + 31) >> 5;  // target slots in use (1..T)
        Layout L;
        {
            const int kl = gc - 32 * (tn - 1);  // targets of the last slot
            L.split = (T <= 4) && (kl <= kSplitMax);
            L.nf = L.split ? tn - 1 : tn;
            L.lg = L.split ? (kl > 1 ? 32 - __clz(kl - 1) : 0) : 5;
        }
        const int lmask = (1 << L.lg) - 1;

        float xi[T], yi[T], zi[T], mi[T];
        unsigned int lo0 = 0xffffffffu, lo1 = 0xffffffffu, lo2 = 0xffffffffu, hi0 = 0u, hi1 = 0u, hi2 = 0u;
#pragma unroll
        for (int t = 0; t < T; t++) {
            const int o = t * 32 + ((L.split && t == L.nf) ? (lane & lmask) : lane);
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (o < gc) {
                q = P.pos_s[gb + o];
                lo0 = min(lo0, bh_f2ord(q.x)); lo1 = min(lo1, bh_f2ord(q.y)); lo2 = min(lo2, bh_f2ord(q.z));
                hi0 = max(hi0, bh_f2ord(q.x)); hi1 = max(hi1, bh_f2ord(q.y)); hi2 = max(hi2, bh_f2ord(q.z));
            }
            xi[t] = q.x; yi[t] = q.y; zi[t] = q.z; mi[t] = q.w;
        }
        {
            const float bx0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo0));
            const float by0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo1));
            const float bz0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo2));
            const float bx1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi0));
            const float by1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi1));
            const float bz1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi2));
            if (lane == 0) {
                S.gbox[0] = bx0; S.gbox[1] = by0; S.gbox[2] = bz0;
                S.gbox[4] = bx1; S.gbox[5] = by1; S.gbox[6] = bz1;
                // half diagonal (a feature of the learned criterion)
                S.gbox[3] = LEARNED ? 0.5f * sqrtf((bx1 - bx0) * (bx1 - bx0) + (by1 - by0) * (by1 - by0) +
                                                   (bz1 - bz0) * (bz1 - bz0))
                                    : 0.0f;
            }
            __syncwarp();
        }

        Acc<T> A;
#if BH_KAHAN_SMEM
        A.kc = kcol;
#endif
#pragma unroll
        for (int t = 0; t < T; t++) {
            A.x[t] = A.y[t] = A.z[t] = A.p[t] = 0.0f;
            A.c(t, 0) = A.c(t, 1) = A.c(t, 2) = A.c(t, 3) = 0.0f;
        }
        bh_eval_self<T>(gc, L, eps2, xi, yi, zi, mi, A);
        Tgt<T> X;
#pragma unroll
        for (int t = 0; t < T; t++) {
            X.x[t] = make_float2(xi[t], xi[t]);
            X.y[t] = make_float2(yi[t], yi[t]);
            X.z[t] = make_float2(zi[t], zi[t]);
        }
        const f2 eps2v = make_float2(eps2, eps2);
        unsigned int g_pc = 0u, g_pp = 0u;  // accepted nodes, particles of opened leaves

        int sp = 1, ring_head = 0, ring_cnt = 0, q_head = 0, q_cnt = 0;
        // root of the group's system: the last level-0 node starting at or before gb
        // (one root per system; a single system has just node 0)
        int root = 0;
        for (int hi = n_roots; hi - root > 1;) {
            const int mid = (root + hi) >> 1;
            if (P.rec[mid].x <= gb) root = mid;
            else hi = mid;
        }
        if (lane == 0) S.stack[0] = (uint32_t)root << 3;
        __syncwarp();
        bool overflow = false;
        while (sp > 0) {
            // ---- pop the top 32 nodes (ranges of siblings)
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

            // ---- test the nodes
            float4 cm = make_float4(0.f, 0.f, 0.f, 0.f);
            float se = 0.f;
            int4 r = make_int4(0, 0, -1, 0);
            if (has) {
                cm = P.com_m[v];
                se = P.seff[v];
                r = P.rec[v];
            }
            const float4 gb0 = bh_lds4(S.gbox), gb1 = bh_lds4(S.gbox + 4);
            const float bx0 = gb0.x, by0 = gb0.y, bz0 = gb0.z, bx1 = gb1.x, by1 = gb1.y, bz1 = gb1.z;
            const float dx = fmaxf(fmaxf(bx0 - cm.x, cm.x - bx1), 0.0f);
            const float dy = fmaxf(fmaxf(by0 - cm.y, cm.y - by1), 0.0f);
            const float dz = fmaxf(fmaxf(bz0 - cm.z, cm.z - bz1), 0.0f);
            const float d2 = bh_dist2(dx, dy, dz);
            const bool member = (r.x < ge) && (r.x + r.y > gb);
            bool acc = has && (d2 > se) && !member;
            if (LEARNED && __ballot_sync(BH_FULL_MASK, acc)) {
                // the guard passed: the network decides (the plain criterion at
                // theta_fb when a feature lies outside the training range)
                // group centre and radius (features of the learned criterion)
                const float gcx = 0.5f * (bx0 + bx1), gcy = 0.5f * (by0 + by1), gcz = 0.5f * (bz0 + bz1);
                const float grg = gb0.w;
                const float4 nf = has ? P.mfeat[v] : make_float4(0.f, 0.f, 0.f, 0.f);
                float f[BH_MLP_NF], side;
                bool inr = bh_mac_features(cm, nf, gcx, gcy, gcz, grg, boxL, f, side);
#pragma unroll
                for (int k = 0; k < BH_MLP_NF; k++) inr = inr && f[k] >= MW->fmin[k] && f[k] <= MW->fmax[k];
                const float yh = bh_mlp_warp(*MW, xs, f);
                const float sfb = fmaxf(sqrtf(se) - side / P.theta_guard, 0.0f) + side / MW->theta_fb;
                acc = acc && (inr ? (yh < MW->ltau) : (d2 > sfb * sfb));
            }
            const bool leaf = has && !acc && (r.z < 0);
            const bool opn = has && !acc && (r.z >= 0);

            // ---- open: push child ranges
            const unsigned int om = __ballot_sync(BH_FULL_MASK, opn);
            const int npush = __popc(om);
            if (sp + npush > kStackCap) {
                overflow = true;
                break;
            }
            if (opn) S.stack[sp + __popc(om & lt)] = ((uint32_t)r.z << 3) | (uint32_t)(r.w - 1);
            sp += npush;

            // ---- accept: cell sources
            const unsigned int am = __ballot_sync(BH_FULL_MASK, acc);
            const int nacc = __popc(am);
            g_pc += (unsigned int)nacc;
            if (ORDER >= 2) {
                if (acc) {
                    const int slot = (q_head + q_cnt + __popc(am & lt)) & (kRing - 1);
                    bh_put_quad(*Q, slot, cm, P.quad[2 * (size_t)v], P.quad[2 * (size_t)v + 1], eps2);
                }
                q_cnt += nacc;
            } else {
                if (acc) bh_put_point(S, (ring_head + ring_cnt + __popc(am & lt)) & (kRing - 1), cm);
                ring_cnt += nacc;
            }

            // ---- rejected leaves: particle ranges outside the group
            const int a0 = r.x, a1 = r.x + r.y;
            const bool pa = leaf && (a0 < gb);
            const bool pb = leaf && (a1 > ge);
            const int pa_n = pa ? (min(a1, gb) - a0) : 0;
            const int pb_s = max(a0, ge);
            const int pb_n = pb ? (a1 - pb_s) : 0;
            const unsigned int ma = __ballot_sync(BH_FULL_MASK, pa), mb = __ballot_sync(BH_FULL_MASK, pb);
            int lq_n = __popc(ma) + __popc(mb);
            if (pa) S.leafq[__popc(ma & lt)] = make_int2(a0, pa_n);
            if (pb) S.leafq[__popc(ma) + __popc(mb & lt)] = make_int2(pb_s, pb_n);
            g_pp += __reduce_add_sync(BH_FULL_MASK, (unsigned int)(pa_n + pb_n));
            __syncwarp();

            // ---- drain: quadrupole tiles, point tiles, particle fills
            if (ORDER >= 2) {
                while (q_cnt >= kTile) {
                    bh_quads<T, WarpQuad, bh_quad_unroll<T, LEARNED>()>(L, *Q, q_head >> 1, eps2v, X, A);
                    q_head ^= kTile;
                    q_cnt -= kTile;
                }
            }
            int lq_pos = 0;
            for (;;) {
                if (ring_cnt >= kTile) {
                    bh_points<T, LEARNED ? kPointUnrollLearned : kPointUnroll>(L, S.ra + (ring_head >> 1), S.rb + (ring_head >> 1),
                                                                        eps2v, X, A);
                    ring_head ^= kTile;
                    ring_cnt -= kTile;
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
                if (lane < nfill)
                    bh_put_point(S, (ring_head + ring_cnt + lane) & (kRing - 1), P.pos_s[S.staging[lane]]);
                ring_cnt += nfill;
                __syncwarp();
            }
        }
        if (overflow) {
            if (lane == 0) bh_set_error(ctrl, BH_ERR_CAPACITY);
            break;
        }
        if (lane == 0) {
            S.tot[0] += ((unsigned long long)g_pp + (unsigned long long)(gc - 1)) * (unsigned long long)gc;
            S.tot[1] += (unsigned long long)g_pc * (unsigned long long)gc;
        }
        // ---- flush the partial tiles (padded with far, massless sources)
        if (ORDER >= 2 && q_cnt > 0) {
            for (int i = lane; i < kTile; i += 32)
                if (i >= q_cnt)
                    bh_put_quad(*Q, q_head + i, bh_pad_source(), make_float4(0.f, 0.f, 0.f, 0.f),
                                make_float4(0.f, 0.f, 0.f, 0.f), eps2);
            __syncwarp();
            bh_quads<T, WarpQuad, bh_quad_unroll<T, LEARNED>()>(L, *Q, q_head >> 1, eps2v, X, A,
                                                                             (q_cnt + 1) >> 1);
        }
        if (ring_cnt > 0) {
            for (int i = lane; i < kTile; i += 32)
                if (i >= ring_cnt) bh_put_point(S, ring_head + i, bh_pad_source());
            __syncwarp();
            constexpr int PU = LEARNED ? kPointUnrollLearned : kPointUnroll;
            bh_points<T, PU>(L, S.ra + (ring_head >> 1), S.rb + (ring_head >> 1), eps2v, X, A,
                             (((ring_cnt + 1) >> 1) + PU - 1) / PU * PU);
        }
        __syncwarp();
        // ---- write (ax, ay, az, phi) in the caller's order; a split slot first
        // adds its phases' sums (lanes l, l + m, l + 2m, ... hold target l)
#pragma unroll
        for (int t = 0; t < T; t++) {
            float4 f = make_float4(A.x[t] - A.c(t, 0), A.y[t] - A.c(t, 1), A.z[t] - A.c(t, 2), A.p[t] - A.c(t, 3));
            if (L.split && t == L.nf) {
                for (int off = 1 << L.lg; off < 32; off <<= 1) {
                    f.x += __shfl_xor_sync(BH_FULL_MASK, f.x, off);
                    f.y += __shfl_xor_sync(BH_FULL_MASK, f.y, off);
                    f.z += __shfl_xor_sync(BH_FULL_MASK, f.z, off);
                    f.w += __shfl_xor_sync(BH_FULL_MASK, f.w, off);
                }
            }
            const int o = t * 32 + lane;
            if (o < gc) P.out[P.perm[gb + o]] = f;
        }
    }
    if (lane == 0) {
        const unsigned long long cnt_pp = S.tot[0], cnt_pc = S.tot[1];
        atomicAdd(&ctrl->n_pp, cnt_pp);
        atomicAdd(&ctrl->n_pc, cnt_pc);
        atomicAdd(&ctrl->cum_pp, cnt_pp);
        atomicAdd(&ctrl->cum_pc, cnt_pc);
    }
}

// ------------------------------------------------------------ warp-specialised walk
// The same walk and the same tiles, split between two warps of a pair: the
// walker warp tests nodes, builds the source tiles and hands each full tile
// to its evaluator warp through a ring of kWsSlots shared-memory slots; the
// evaluator holds the group's targets and applies the tiles in the order they
// were handed over, which is the order of the one-warp kernel, so the results
// are the same bits.  While an evaluator works through a tile its walker
// already builds the next ones.  Slots are guarded by mbarriers (one "full",
// one "empty" per slot, 32 arrivals each); every wait is bounded and gives up
// with BH_ERR_DEVICE_TIMEOUT.  A block holds four pairs: warps 0-3 walk,
// warps 4-7 evaluate.  On a 16M-particle clumpy set this kernel is slower than
// the one-warp kernel: there the other warps' evaluation already hides the
// walk, and two evaluator warps per scheduler issue less of it than four
// mixed warps.  It is selected only on request (walk_variant).
#ifndef BH_WS_SLOTS
#define BH_WS_SLOTS 4
#endif
constexpr int kWsSlots = BH_WS_SLOTS;
constexpr int kWsPairs = 4;
constexpr int kWsSpinLimit = 1 << 22;
constexpr unsigned long long kWsTimeoutNs = 1000000000ull;
enum : int { kWsPoints = 0, kWsQuads = 1, kWsBegin = 2, kWsEnd = 3, kWsExit = 4 };

struct WsTile {  // kTile sources as pairs, laid out as WarpSmem (points: a, b) and WarpQuad (cells: a..f)
    float4 a[kTilePairs], b[kTilePairs], c[kTilePairs], d[kTilePairs], e[kTilePairs], f[kTilePairs];
};
struct WsChannel {
    WsTile tile[kWsSlots];
    int kind[kWsSlots];
    int arg[kWsSlots];
    unsigned long long full[kWsSlots];
    unsigned long long empty[kWsSlots];
};

__device__ __forceinline__ unsigned int bh_smem_addr(const void* p)
{
    return static_cast<unsigned int>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void bh_mbar_init(unsigned long long* b, unsigned int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bh_smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bh_mbar_arrive(unsigned long long* b)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bh_smem_addr(b))
                 : "memory");
}
__device__ __forceinline__ bool bh_mbar_try_wait(unsigned long long* b, unsigned int parity)
{
    unsigned int ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bh_smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// Wait for the phase of the given parity to complete.  False (with the error
// recorded) once a second has passed on the global timer or after
// kWsSpinLimit polls, whichever comes first; false at once when another warp
// has aborted.
__device__ __forceinline__ unsigned long long bh_globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool bh_mbar_wait(unsigned long long* b, unsigned int parity, bh_dev_ctrl* c)
{
    if (bh_mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = bh_globaltimer();
    for (int i = 0; i < kWsSpinLimit; i++) {
        if (bh_mbar_try_wait(b, parity)) return true;
        if ((i & 63) == 63) {
            if (*(volatile unsigned int*)&c->abort) return false;
            if (bh_globaltimer() - t0 > kWsTimeoutNs) break;
        }
    }
    bh_set_error(c, BH_ERR_DEVICE_TIMEOUT);
    return false;
}

// Walker side: claim the next slot (waiting until its evaluator has released
// it), let fill() write the tile, publish it.  False if the wait gave up.
template <class Fill>
__device__ __forceinline__ bool bh_ws_send(WsChannel& C, int& item, int kind, int arg, bh_dev_ctrl* ctrl,
                                           Fill fill)
{
    const int s = item % kWsSlots;
    const unsigned int use = (unsigned int)(item / kWsSlots);
    const bool ok = bh_mbar_wait(&C.empty[s], (use & 1u) ^ 1u, ctrl);
    if (__any_sync(BH_FULL_MASK, !ok)) return false;
    fill(C.tile[s]);
    if ((threadIdx.x & 31) == 0) {
        C.kind[s] = kind;
        C.arg[s] = arg;
    }
    __syncwarp();
    bh_mbar_arrive(&C.full[s]);
    item++;
    return true;
}

template <int T>
__host__ __device__ constexpr int bh_ws_min_blocks() { return T <= 1 ? 3 : 2; }

template <int T, int ORDER>
__global__ void __launch_bounds__(256, bh_ws_min_blocks<T>()) bh_walk_ws_kernel(WalkParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int pair = wib & (kWsPairs - 1);
    const bool walker = wib < kWsPairs;
    WsChannel& C = reinterpret_cast<WsChannel*>(smem_raw)[pair];
    unsigned char* base = smem_raw + kWsPairs * sizeof(WsChannel);
    WarpSmem& S = reinterpret_cast<WarpSmem*>(base)[pair];
    base += kWsPairs * sizeof(WarpSmem);
    WarpQuad* Q = nullptr;
    if (ORDER >= 2) {
        Q = reinterpret_cast<WarpQuad*>(base) + pair;
        base += kWsPairs * sizeof(WarpQuad);
    }
    float* kcol = reinterpret_cast<float*>(base + (size_t)pair * bh_kahan_smem_bytes<T>()) + lane;
    if (walker && lane < kWsSlots) {
        bh_mbar_init(&C.full[lane], 32u);
        bh_mbar_init(&C.empty[lane], 32u);
    }
    __syncthreads();

    const unsigned int lt = bh_lanemask_lt();
    const float eps2 = P.eps2;
    bh_dev_ctrl* ctrl = P.ctrl;
    int item = 0;

    if (walker) {
        const int ng = (int)ctrl->n_groups;
        const int n_roots = (int)ctrl->level_offset[1];
        unsigned long long cnt_pp = 0ull, cnt_pc = 0ull;
        bool alive = true;
        auto send_quads = [&](int p0) {
            return bh_ws_send(C, item, kWsQuads, 0, ctrl, [&](WsTile& t) {
                if (lane < kTilePairs) {
                    t.a[lane] = Q->a[p0 + lane]; t.b[lane] = Q->b[p0 + lane]; t.c[lane] = Q->c[p0 + lane];
                    t.d[lane] = Q->d[p0 + lane]; t.e[lane] = Q->e[p0 + lane]; t.f[lane] = Q->f[p0 + lane];
                }
            });
        };
        auto send_points = [&](int p0) {
            return bh_ws_send(C, item, kWsPoints, 0, ctrl, [&](WsTile& t) {
                if (lane < kTilePairs) {
                    t.a[lane] = S.ra[p0 + lane];
                    t.b[lane] = S.rb[p0 + lane];
                }
            });
        };
        auto no_tile = [](WsTile&) {};
        for (;;) {
            int g = 0;
            if (lane == 0) g = (int)atomicAdd(&ctrl->group_ctr, 1u);
            g = __shfl_sync(BH_FULL_MASK, g, 0);
            if (g >= ng) break;
            int ab = 0;
            if (lane == 0) ab = (int)*(volatile unsigned int*)&ctrl->abort;
            if (__shfl_sync(BH_FULL_MASK, ab, 0)) break;
            const int gb = P.g_first[g], gc = P.g_count[g], ge = gb + gc;
            unsigned int lo0 = 0xffffffffu, lo1 = 0xffffffffu, lo2 = 0xffffffffu, hi0 = 0u, hi1 = 0u, hi2 = 0u;
            for (int o = lane; o < gc; o += 32) {
                const float4 q = P.pos_s[gb + o];
                lo0 = min(lo0, bh_f2ord(q.x)); lo1 = min(lo1, bh_f2ord(q.y)); lo2 = min(lo2, bh_f2ord(q.z));
                hi0 = max(hi0, bh_f2ord(q.x)); hi1 = max(hi1, bh_f2ord(q.y)); hi2 = max(hi2, bh_f2ord(q.z));
            }
            const float bx0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo0));
            const float by0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo1));
            const float bz0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo2));
            const float bx1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi0));
            const float by1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi1));
            const float bz1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi2));
            if (!(alive = bh_ws_send(C, item, kWsBegin, g, ctrl, no_tile))) break;
            cnt_pp += (unsigned long long)gc * (unsigned long long)(gc - 1);

            int sp = 1, ring_head = 0, ring_cnt = 0, q_head = 0, q_cnt = 0;
            int root = 0;
            for (int hi = n_roots; hi - root > 1;) {
                const int mid = (root + hi) >> 1;
                if (P.rec[mid].x <= gb) root = mid;
                else hi = mid;
            }
            if (lane == 0) S.stack[0] = (uint32_t)root << 3;
            __syncwarp();
            bool overflow = false;
            while (sp > 0 && alive) {
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

                float4 cm = make_float4(0.f, 0.f, 0.f, 0.f);
                float se = 0.f;
                int4 r = make_int4(0, 0, -1, 0);
                if (has) {
                    cm = P.com_m[v];
                    se = P.seff[v];
                    r = P.rec[v];
                }
                const float dx = fmaxf(fmaxf(bx0 - cm.x, cm.x - bx1), 0.0f);
                const float dy = fmaxf(fmaxf(by0 - cm.y, cm.y - by1), 0.0f);
                const float dz = fmaxf(fmaxf(bz0 - cm.z, cm.z - bz1), 0.0f);
                const float d2 = bh_dist2(dx, dy, dz);
                const bool member = (r.x < ge) && (r.x + r.y > gb);
                const bool acc = has && (d2 > se) && !member;
                const bool leaf = has && !acc && (r.z < 0);
                const bool opn = has && !acc && (r.z >= 0);

                const unsigned int om = __ballot_sync(BH_FULL_MASK, opn);
                const int npush = __popc(om);
                if (sp + npush > kStackCap) {
                    overflow = true;
                    break;
                }
                if (opn) S.stack[sp + __popc(om & lt)] = ((uint32_t)r.z << 3) | (uint32_t)(r.w - 1);
                sp += npush;

                const unsigned int am = __ballot_sync(BH_FULL_MASK, acc);
                const int nacc = __popc(am);
                cnt_pc += (unsigned long long)nacc * (unsigned long long)gc;
                if (ORDER >= 2) {
                    if (acc) {
                        const int slot = (q_head + q_cnt + __popc(am & lt)) & (kRing - 1);
                        bh_put_quad(*Q, slot, cm, P.quad[2 * (size_t)v], P.quad[2 * (size_t)v + 1], eps2);
                    }
                    q_cnt += nacc;
                } else {
                    if (acc) bh_put_point(S, (ring_head + ring_cnt + __popc(am & lt)) & (kRing - 1), cm);
                    ring_cnt += nacc;
                }

                const int a0 = r.x, a1 = r.x + r.y;
                const bool pa = leaf && (a0 < gb);
                const bool pb = leaf && (a1 > ge);
                const int pa_n = pa ? (min(a1, gb) - a0) : 0;
                const int pb_s = max(a0, ge);
                const int pb_n = pb ? (a1 - pb_s) : 0;
                const unsigned int ma = __ballot_sync(BH_FULL_MASK, pa), mb = __ballot_sync(BH_FULL_MASK, pb);
                int lq_n = __popc(ma) + __popc(mb);
                if (pa) S.leafq[__popc(ma & lt)] = make_int2(a0, pa_n);
                if (pb) S.leafq[__popc(ma) + __popc(mb & lt)] = make_int2(pb_s, pb_n);
                cnt_pp += (unsigned long long)__reduce_add_sync(BH_FULL_MASK, (unsigned int)(pa_n + pb_n)) *
                          (unsigned long long)gc;
                __syncwarp();

                if (ORDER >= 2) {
                    while (q_cnt >= kTile && alive) {
                        __syncwarp();
                        alive = send_quads(q_head >> 1);
                        q_head ^= kTile;
                        q_cnt -= kTile;
                    }
                }
                int lq_pos = 0;
                while (alive) {
                    if (ring_cnt >= kTile) {
                        __syncwarp();
                        alive = send_points(ring_head >> 1);
                        ring_head ^= kTile;
                        ring_cnt -= kTile;
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
                    if (lane < nfill)
                        bh_put_point(S, (ring_head + ring_cnt + lane) & (kRing - 1), P.pos_s[S.staging[lane]]);
                    ring_cnt += nfill;
                    __syncwarp();
                }
            }
            if (!alive) break;
            if (overflow) {
                if (lane == 0) bh_set_error(ctrl, BH_ERR_CAPACITY);
                break;
            }
            // flush the partial tiles (padded with far, massless sources), then close the group
            if (ORDER >= 2 && q_cnt > 0) {
                for (int i = lane; i < kTile; i += 32)
                    if (i >= q_cnt)
                        bh_put_quad(*Q, q_head + i, bh_pad_source(), make_float4(0.f, 0.f, 0.f, 0.f),
                                    make_float4(0.f, 0.f, 0.f, 0.f), eps2);
                __syncwarp();
                if (!(alive = send_quads(q_head >> 1))) break;
            }
            if (ring_cnt > 0) {
                for (int i = lane; i < kTile; i += 32)
                    if (i >= ring_cnt) bh_put_point(S, ring_head + i, bh_pad_source());
                __syncwarp();
                if (!(alive = send_points(ring_head >> 1))) break;
            }
            if (!(alive = bh_ws_send(C, item, kWsEnd, g, ctrl, no_tile))) break;
        }
        if (alive) bh_ws_send(C, item, kWsExit, 0, ctrl, no_tile);
        if (lane == 0) {
            atomicAdd(&ctrl->n_pp, cnt_pp);
            atomicAdd(&ctrl->n_pc, cnt_pc);
            atomicAdd(&ctrl->cum_pp, cnt_pp);
            atomicAdd(&ctrl->cum_pc, cnt_pc);
        }
        return;
    }

    // ---- evaluator
    const f2 eps2v = make_float2(eps2, eps2);
    int gb = 0, gc = 0;
    Layout L;
    L.nf = 1; L.split = false; L.lg = 5;
    float xi[T], yi[T], zi[T], mi[T];
    Tgt<T> X;
    Acc<T> A;
#if BH_KAHAN_SMEM
    A.kc = kcol;
#endif
    for (;;) {
        const int s = item % kWsSlots;
        const unsigned int use = (unsigned int)(item / kWsSlots);
        const bool ok = bh_mbar_wait(&C.full[s], use & 1u, ctrl);
        if (__any_sync(BH_FULL_MASK, !ok)) break;
        const int kind = C.kind[s];
        if (kind == kWsExit) break;
        if (kind == kWsBegin) {
            const int g = C.arg[s];
            gb = P.g_first[g];
            gc = P.g_count[g];
            const int tn = (gc + 31) >> 5;
            const int kl = gc - 32 * (tn - 1);
            L.split = (T <= 4) && (kl <= kSplitMax);
            L.nf = L.split ? tn - 1 : tn;
            L.lg = L.split ? (kl > 1 ? 32 - __clz(kl - 1) : 0) : 5;
            const int lmask = (1 << L.lg) - 1;
#pragma unroll
            for (int t = 0; t < T; t++) {
                const int o = t * 32 + ((L.split && t == L.nf) ? (lane & lmask) : lane);
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (o < gc) q = P.pos_s[gb + o];
                xi[t] = q.x; yi[t] = q.y; zi[t] = q.z; mi[t] = q.w;
            }
#pragma unroll
            for (int t = 0; t < T; t++) {
                A.x[t] = A.y[t] = A.z[t] = A.p[t] = 0.0f;
                A.c(t, 0) = A.c(t, 1) = A.c(t, 2) = A.c(t, 3) = 0.0f;
            }
            bh_eval_self<T>(gc, L, eps2, xi, yi, zi, mi, A);
#pragma unroll
            for (int t = 0; t < T; t++) {
                X.x[t] = make_float2(xi[t], xi[t]);
                X.y[t] = make_float2(yi[t], yi[t]);
                X.z[t] = make_float2(zi[t], zi[t]);
            }
        } else if (kind == kWsQuads) {
            if (ORDER >= 2) bh_quads<T, WsTile, kQuadUnrollPaired>(L, C.tile[s], 0, eps2v, X, A);
        } else if (kind == kWsPoints) {
            bh_points<T, kPointUnrollPaired>(L, C.tile[s].a, C.tile[s].b, eps2v, X, A);
        } else if (kind == kWsEnd) {
#pragma unroll
            for (int t = 0; t < T; t++) {
                float4 f = make_float4(A.x[t] - A.c(t, 0), A.y[t] - A.c(t, 1), A.z[t] - A.c(t, 2), A.p[t] - A.c(t, 3));
                if (L.split && t == L.nf) {
                    for (int off = 1 << L.lg; off < 32; off <<= 1) {
                        f.x += __shfl_xor_sync(BH_FULL_MASK, f.x, off);
                        f.y += __shfl_xor_sync(BH_FULL_MASK, f.y, off);
                        f.z += __shfl_xor_sync(BH_FULL_MASK, f.z, off);
                        f.w += __shfl_xor_sync(BH_FULL_MASK, f.w, off);
                    }
                }
                const int o = t * 32 + lane;
                if (o < gc) P.out[P.perm[gb + o]] = f;
            }
        }
        __syncwarp();
        bh_mbar_arrive(&C.empty[s]);
        item++;
    }
}

template <int T, int ORDER>
static int bh_walk_ws_launch(const WalkParams& P, int sm_count, cudaStream_t s)
{
    const size_t smem = kWsPairs * (sizeof(WsChannel) + sizeof(WarpSmem) + (ORDER >= 2 ? sizeof(WarpQuad) : 0) +
                                    bh_kahan_smem_bytes<T>());
    auto kern = bh_walk_ws_kernel<T, ORDER>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return BH_ERR_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, smem) != cudaSuccess || bps < 1) bps = 1;
    kern<<<sm_count * bps, 256, smem, s>>>(P);
    return BH_OK;
}

// ------------------------------------------------------------ TMA-staged walk
// The one-warp walk with its memory traffic moved onto bulk asynchronous
// copies (cp.async.bulk, global -> this CTA's shared memory, completed on an
// mbarrier):
//   * node tiles: each popped range of siblings is one copy of its walk
//     records (centre of mass and mass, first/count/children/S_eff, the
//     quadrupole) into the warp's node landing area, record i of the pop at
//     slot i; the next pop is taken and its copies issued as soon as this
//     pop's pushes are done, so they land while this pop's tiles are
//     evaluated;
//   * particle tiles: the particles of a pop's rejected leaves (up to 128 per
//     round) are one copy per leaf range into the particle landing area,
//     issued with the next pop's node copies, before the pop's quadrupole
//     tiles are evaluated; the point ring is then filled from the landing
//     area in the same 32-particle slices as the one-warp kernel's.
// The landed records are converted into the same negated pair rings, in the
// same order, as the one-warp kernel's, so the tiles and the results are the
// same bits.  Waits are bounded (BH_ERR_DEVICE_TIMEOUT); every copy reads
// this GPU's own memory and lands in this CTA's shared memory.
__device__ __forceinline__ void bh_mbar_expect_tx(unsigned long long* b, unsigned int bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     bh_smem_addr(b)),
                 "r"(bytes)
                 : "memory");
}
// bytes (a multiple of 16) from global src to shared dst, both 16-byte aligned
__device__ __forceinline__ void bh_bulk_g2s(void* dst, const void* src, unsigned int bytes, unsigned long long* b)
{
    asm volatile("cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     bh_smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(bh_smem_addr(b))
                 : "memory");
}
// order this thread's earlier generic-proxy accesses of shared memory before
// its later async-proxy ones (a landing area is refilled after it was read)
__device__ __forceinline__ void bh_fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Wait for this warp's own copies: no early exit on another warp's abort
// (copies of valid addresses always complete); false after a second on the
// global timer or kWsSpinLimit polls, with BH_ERR_DEVICE_TIMEOUT recorded.
__device__ __forceinline__ bool bh_mbar_wait_own(unsigned long long* b, unsigned int parity, bh_dev_ctrl* c)
{
    if (bh_mbar_try_wait(b, parity)) return true;
    const unsigned long long t0 = bh_globaltimer();
    for (int i = 0; i < kWsSpinLimit; i++) {
        if (bh_mbar_try_wait(b, parity)) return true;
        if ((i & 63) == 63 && bh_globaltimer() - t0 > kWsTimeoutNs) break;
    }
    bh_set_error(c, BH_ERR_DEVICE_TIMEOUT);
    return false;
}

// Particles of rejected leaves landed per round of copies (a multiple of 32).
#ifndef BH_TMA_PART_CAP
#define BH_TMA_PART_CAP 128
#endif
constexpr int kTmaPartCap = BH_TMA_PART_CAP;

template <int ORDER>
struct TmaLanding {
    float4 node[32 * bh_wrec_f4(ORDER)];  // the pop's walk records, record i at slot i
    float4 part[kTmaPartCap];              // a round of particles of rejected leaves
    unsigned long long bar_node, bar_part;
};

template <int T, int ORDER>
__global__ void __launch_bounds__(128, bh_walk_min_blocks<T, false>()) bh_walk_tma_kernel(WalkParams P)
{
    constexpr int RF = bh_wrec_f4(ORDER);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    WarpSmem& S = reinterpret_cast<WarpSmem*>(smem_raw)[wib];
    unsigned char* base = smem_raw + (size_t)nwarps * sizeof(WarpSmem);
    WarpQuad* Q = nullptr;
    if (ORDER >= 2) {
        Q = reinterpret_cast<WarpQuad*>(base) + wib;
        base += (size_t)nwarps * sizeof(WarpQuad);
    }
    TmaLanding<ORDER>& LD = reinterpret_cast<TmaLanding<ORDER>*>(base)[wib];
    base += (size_t)nwarps * sizeof(TmaLanding<ORDER>);
    float* kcol = reinterpret_cast<float*>(base + (size_t)wib * bh_kahan_smem_bytes<T>()) + lane;
    if (lane == 0) {
        bh_mbar_init(&LD.bar_node, 1u);
        bh_mbar_init(&LD.bar_part, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    unsigned int ph_node = 0u, ph_part = 0u;      // phases to wait for next
    bool node_out = false, part_out = false;      // a copy batch is in flight (warp-uniform)

    const unsigned int lt = bh_lanemask_lt();
    const float eps2 = P.eps2;
    bh_dev_ctrl* ctrl = P.ctrl;
    const int ng = (int)ctrl->n_groups;
    const int n_roots = (int)ctrl->level_offset[1];
    if (lane == 0) S.tot[0] = S.tot[1] = 0ull;
    bool alive = true;

    for (;;) {
        int g = 0;
        if (lane == 0) g = (int)atomicAdd(&ctrl->group_ctr, 1u);
        g = __shfl_sync(BH_FULL_MASK, g, 0);
        if (g >= ng) break;
        int ab = 0;
        if (lane == 0) ab = (int)*(volatile unsigned int*)&ctrl->abort;
        if (__shfl_sync(BH_FULL_MASK, ab, 0)) break;
        const int gb = P.g_first[g], gc = P.g_count[g], ge = gb + gc;
        const int tn = (gc + 31) >> 5;
        Layout L;
        {
            const int kl = gc - 32 * (tn - 1);
            L.split = (T <= 4) && (kl <= kSplitMax);
            L.nf = L.split ? tn - 1 : tn;
            L.lg = L.split ? (kl > 1 ? 32 - __clz(kl - 1) : 0) : 5;
        }
        const int lmask = (1 << L.lg) - 1;

        float xi[T], yi[T], zi[T], mi[T];
        unsigned int lo0 = 0xffffffffu, lo1 = 0xffffffffu, lo2 = 0xffffffffu, hi0 = 0u, hi1 = 0u, hi2 = 0u;
#pragma unroll
        for (int t = 0; t < T; t++) {
            const int o = t * 32 + ((L.split && t == L.nf) ? (lane & lmask) : lane);
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (o < gc) {
                q = P.pos_s[gb + o];
                lo0 = min(lo0, bh_f2ord(q.x)); lo1 = min(lo1, bh_f2ord(q.y)); lo2 = min(lo2, bh_f2ord(q.z));
                hi0 = max(hi0, bh_f2ord(q.x)); hi1 = max(hi1, bh_f2ord(q.y)); hi2 = max(hi2, bh_f2ord(q.z));
            }
            xi[t] = q.x; yi[t] = q.y; zi[t] = q.z; mi[t] = q.w;
        }
        {
            const float bx0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo0));
            const float by0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo1));
            const float bz0 = bh_ord2f(__reduce_min_sync(BH_FULL_MASK, lo2));
            const float bx1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi0));
            const float by1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi1));
            const float bz1 = bh_ord2f(__reduce_max_sync(BH_FULL_MASK, hi2));
            if (lane == 0) {
                S.gbox[0] = bx0; S.gbox[1] = by0; S.gbox[2] = bz0; S.gbox[3] = 0.0f;
                S.gbox[4] = bx1; S.gbox[5] = by1; S.gbox[6] = bz1;
            }
            __syncwarp();
        }

        Acc<T> A;
#if BH_KAHAN_SMEM
        A.kc = kcol;
#endif
#pragma unroll
        for (int t = 0; t < T; t++) {
            A.x[t] = A.y[t] = A.z[t] = A.p[t] = 0.0f;
            A.c(t, 0) = A.c(t, 1) = A.c(t, 2) = A.c(t, 3) = 0.0f;
        }
        bh_eval_self<T>(gc, L, eps2, xi, yi, zi, mi, A);
        Tgt<T> X;
#pragma unroll
        for (int t = 0; t < T; t++) {
            X.x[t] = make_float2(xi[t], xi[t]);
            X.y[t] = make_float2(yi[t], yi[t]);
            X.z[t] = make_float2(zi[t], zi[t]);
        }
        const f2 eps2v = make_float2(eps2, eps2);
        unsigned int g_pc = 0u, g_pp = 0u;

        int sp = 1, ring_head = 0, ring_cnt = 0, q_head = 0, q_cnt = 0;
        int root = 0;
        for (int hi = n_roots; hi - root > 1;) {
            const int mid = (root + hi) >> 1;
            if (P.rec[mid].x <= gb) root = mid;
            else hi = mid;
        }
        if (lane == 0) S.stack[0] = (uint32_t)root << 3;
        __syncwarp();

        // Pop the top 32 nodes (ranges of siblings) and issue one copy of
        // walk records per range; returns the number of nodes popped.
        auto pop_issue = [&]() -> int {
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
            const bool full = (lane < sp) && (take == c);
            const int nfull = __popc(__ballot_sync(BH_FULL_MASK, full));
            const int npop = min(__shfl_sync(BH_FULL_MASK, incl, 31), 32);
            __syncwarp();
            if (lane == nfull && lane < sp && take > 0)
                S.stack[sp - 1 - lane] = ((uint32_t)(st + take) << 3) | (uint32_t)(c - take - 1);
            sp -= nfull;
            if (npop > 0) {
                // the expected bytes are the sum of the ranges' copies (sum of take = npop)
                bh_fence_proxy_async();
                if (lane == 0) bh_mbar_expect_tx(&LD.bar_node, (unsigned int)(npop * RF * 16));
                __syncwarp();
                if (take > 0)
                    bh_bulk_g2s(&LD.node[excl * RF], P.wrec + (size_t)st * RF, (unsigned int)(take * RF * 16),
                                &LD.bar_node);
                node_out = true;
            }
            __syncwarp();
            return npop;
        };
        // Take the next round of up to kTmaPartCap particles from the pending
        // leaf ranges at lq_pos (at most 32 ranges) and issue their copies;
        // returns the round's particle count.
        auto round_issue = [&](int& lq_pos, int lq_n) -> int {
            int c2 = 0;
            int2 q = make_int2(0, 0);
            if (lq_pos + lane < lq_n) {
                q = S.leafq[lq_pos + lane];
                c2 = q.y;
            }
            const int inc2 = bh_warp_incl_scan(c2);
            const int ex2 = inc2 - c2;
            const int take2 = max(0, min(c2, kTmaPartCap - ex2));
            const bool full2 = (lq_pos + lane < lq_n) && (take2 == c2);
            const int nf2 = __popc(__ballot_sync(BH_FULL_MASK, full2));
            const int nround = min(__shfl_sync(BH_FULL_MASK, inc2, 31), kTmaPartCap);
            __syncwarp();
            if (lane == nf2 && lq_pos + lane < lq_n && take2 > 0)
                S.leafq[lq_pos + lane] = make_int2(q.x + take2, c2 - take2);
            lq_pos += nf2;
            // ranges that continue the previous lane's range (sibling leaves are
            // contiguous in particle order, and so are their landing slots)
            // join its copy: one copy per run of contiguous ranges
            const int prev_end = __shfl_up_sync(BH_FULL_MASK, q.x + take2, 1);
            const bool cont = lane > 0 && take2 > 0 && q.x == prev_end;
            const unsigned int cm = __ballot_sync(BH_FULL_MASK, cont);
            const unsigned int after = (lane < 31) ? (~cm & (0xffffffffu << (lane + 1))) : 0u;
            const int next = after ? __ffs(after) - 1 : 32;
            const int ex_next = __shfl_sync(BH_FULL_MASK, ex2, next & 31);
            const int run = (next < 32 ? min(ex_next, nround) : nround) - ex2;
            bh_fence_proxy_async();
            if (lane == 0) bh_mbar_expect_tx(&LD.bar_part, (unsigned int)(nround * 16));
            __syncwarp();
            if (take2 > 0 && !cont)
                bh_bulk_g2s(&LD.part[ex2], P.pos_s + q.x, (unsigned int)(run * 16), &LD.bar_part);
            part_out = true;
            __syncwarp();
            return nround;
        };

        bool overflow = false;
        int npop = pop_issue();
        while (npop > 0) {
            // ---- the pop's records have landed: test the nodes
            if (!(alive = __all_sync(BH_FULL_MASK, bh_mbar_wait_own(&LD.bar_node, ph_node, ctrl)))) break;
            ph_node ^= 1u;
            node_out = false;
            const bool has = lane < npop;
            float4 cm = make_float4(0.f, 0.f, 0.f, 0.f), qa = cm, qb = cm;
            int rfirst = 0, rcount = 0, rchn = -1;
            float se = 0.f;
            if (has) {
                cm = LD.node[lane * RF];
                const float4 w1 = LD.node[lane * RF + 1];
                rfirst = __float_as_int(w1.x);
                rcount = __float_as_int(w1.y);
                rchn = __float_as_int(w1.z);
                se = w1.w;
                if (ORDER >= 2) {
                    qa = LD.node[lane * RF + 2];
                    qb = LD.node[lane * RF + 3];
                }
            }
            const float4 gb0 = bh_lds4(S.gbox), gb1 = bh_lds4(S.gbox + 4);
            const float dx = fmaxf(fmaxf(gb0.x - cm.x, cm.x - gb1.x), 0.0f);
            const float dy = fmaxf(fmaxf(gb0.y - cm.y, cm.y - gb1.y), 0.0f);
            const float dz = fmaxf(fmaxf(gb0.z - cm.z, cm.z - gb1.z), 0.0f);
            const float d2 = bh_dist2(dx, dy, dz);
            const bool member = (rfirst < ge) && (rfirst + rcount > gb);
            const bool acc = has && (d2 > se) && !member;
            const bool leaf = has && !acc && (rchn < 0);
            const bool opn = has && !acc && (rchn >= 0);

            // ---- open: push child ranges
            const unsigned int om = __ballot_sync(BH_FULL_MASK, opn);
            const int npush = __popc(om);
            if (sp + npush > kStackCap) {
                overflow = true;
                break;
            }
            if (opn) S.stack[sp + __popc(om & lt)] = (uint32_t)rchn;
            sp += npush;

            // ---- accept: cell sources (records already in registers)
            const unsigned int am = __ballot_sync(BH_FULL_MASK, acc);
            const int nacc = __popc(am);
            g_pc += (unsigned int)nacc;
            if (ORDER >= 2) {
                if (acc) bh_put_quad(*Q, (q_head + q_cnt + __popc(am & lt)) & (kRing - 1), cm, qa, qb, eps2);
                q_cnt += nacc;
            } else {
                if (acc) bh_put_point(S, (ring_head + ring_cnt + __popc(am & lt)) & (kRing - 1), cm);
                ring_cnt += nacc;
            }

            // ---- rejected leaves: particle ranges outside the group
            const int a0 = rfirst, a1 = rfirst + rcount;
            const bool pa = leaf && (a0 < gb);
            const bool pb = leaf && (a1 > ge);
            const int pa_n = pa ? (min(a1, gb) - a0) : 0;
            const int pb_s = max(a0, ge);
            const int pb_n = pb ? (a1 - pb_s) : 0;
            const unsigned int ma = __ballot_sync(BH_FULL_MASK, pa), mb = __ballot_sync(BH_FULL_MASK, pb);
            const int lq_n = __popc(ma) + __popc(mb);
            if (pa) S.leafq[__popc(ma & lt)] = make_int2(a0, pa_n);
            if (pb) S.leafq[__popc(ma) + __popc(mb & lt)] = make_int2(pb_s, pb_n);
            g_pp += __reduce_add_sync(BH_FULL_MASK, (unsigned int)(pa_n + pb_n));
            __syncwarp();

            // ---- the next pop: its records land while this pop's tiles run
            npop = pop_issue();
            int lq_pos = 0, pbase = 0, pavail = 0;
            bool pending = false;
            if (lq_pos < lq_n) {
                pavail = round_issue(lq_pos, lq_n);
                pending = true;
            }

            // ---- drain: quadrupole tiles, then point tiles fed from the landed rounds
            if (ORDER >= 2) {
                while (q_cnt >= kTile) {
                    bh_quads<T, WarpQuad, kQuadUnrollTma>(L, *Q, q_head >> 1, eps2v, X, A);
                    q_head ^= kTile;
                    q_cnt -= kTile;
                }
            }
            for (;;) {
                if (ring_cnt >= kTile) {
                    bh_points<T, kPointUnroll>(L, S.ra + (ring_head >> 1), S.rb + (ring_head >> 1), eps2v, X, A);
                    ring_head ^= kTile;
                    ring_cnt -= kTile;
                    continue;
                }
                if (pbase < pavail) {
                    if (pending) {
                        if (!(alive = __all_sync(BH_FULL_MASK, bh_mbar_wait_own(&LD.bar_part, ph_part, ctrl))))
                            break;
                        ph_part ^= 1u;
                        part_out = false;
                        pending = false;
                    }
                    const int nfill = min(32, pavail - pbase);
                    if (lane < nfill)
                        bh_put_point(S, (ring_head + ring_cnt + lane) & (kRing - 1), LD.part[pbase + lane]);
                    ring_cnt += nfill;
                    pbase += nfill;
                    __syncwarp();
                    continue;
                }
                if (lq_pos < lq_n) {
                    pavail = round_issue(lq_pos, lq_n);
                    pbase = 0;
                    pending = true;
                    continue;
                }
                break;
            }
            if (!alive) break;
        }
        if (!alive) break;
        if (overflow) {
            // the next pop was not issued (the loop ended at the push); nothing is in flight
            if (lane == 0) bh_set_error(ctrl, BH_ERR_CAPACITY);
            break;
        }
        if (lane == 0) {
            S.tot[0] += ((unsigned long long)g_pp + (unsigned long long)(gc - 1)) * (unsigned long long)gc;
            S.tot[1] += (unsigned long long)g_pc * (unsigned long long)gc;
        }
        // ---- flush the partial tiles (padded with far, massless sources)
        if (ORDER >= 2 && q_cnt > 0) {
            for (int i = lane; i < kTile; i += 32)
                if (i >= q_cnt)
                    bh_put_quad(*Q, q_head + i, bh_pad_source(), make_float4(0.f, 0.f, 0.f, 0.f),
                                make_float4(0.f, 0.f, 0.f, 0.f), eps2);
            __syncwarp();
            bh_quads<T, WarpQuad, kQuadUnrollTma>(L, *Q, q_head >> 1, eps2v, X, A, (q_cnt + 1) >> 1);
        }
        if (ring_cnt > 0) {
            for (int i = lane; i < kTile; i += 32)
                if (i >= ring_cnt) bh_put_point(S, ring_head + i, bh_pad_source());
            __syncwarp();
            bh_points<T, kPointUnroll>(L, S.ra + (ring_head >> 1), S.rb + (ring_head >> 1), eps2v, X, A,
                                       (((ring_cnt + 1) >> 1) + kPointUnroll - 1) / kPointUnroll * kPointUnroll);
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < T; t++) {
            float4 f = make_float4(A.x[t] - A.c(t, 0), A.y[t] - A.c(t, 1), A.z[t] - A.c(t, 2), A.p[t] - A.c(t, 3));
            if (L.split && t == L.nf) {
                for (int off = 1 << L.lg; off < 32; off <<= 1) {
                    f.x += __shfl_xor_sync(BH_FULL_MASK, f.x, off);
                    f.y += __shfl_xor_sync(BH_FULL_MASK, f.y, off);
                    f.z += __shfl_xor_sync(BH_FULL_MASK, f.z, off);
                    f.w += __shfl_xor_sync(BH_FULL_MASK, f.w, off);
                }
            }
            const int o = t * 32 + lane;
            if (o < gc) P.out[P.perm[gb + o]] = f;
        }
    }
    // a wait gave up: wait once more (bounded) for copies still in flight
    // into this warp's landing areas before the block's shared memory goes
    if (node_out) bh_mbar_wait_own(&LD.bar_node, ph_node, ctrl);
    if (part_out) bh_mbar_wait_own(&LD.bar_part, ph_part, ctrl);
    if (lane == 0) {
        const unsigned long long cnt_pp = S.tot[0], cnt_pc = S.tot[1];
        atomicAdd(&ctrl->n_pp, cnt_pp);
        atomicAdd(&ctrl->n_pc, cnt_pc);
        atomicAdd(&ctrl->cum_pp, cnt_pp);
        atomicAdd(&ctrl->cum_pc, cnt_pc);
    }
}

template <int T, int ORDER>
static int bh_walk_tma_launch_t(const WalkParams& P, int sm_count, int block_threads, int blocks_per_sm,
                                cudaStream_t s)
{
    const int nw = block_threads / 32;
    const size_t smem = (size_t)nw * (sizeof(WarpSmem) + (ORDER >= 2 ? sizeof(WarpQuad) : 0) +
                                      sizeof(TmaLanding<ORDER>) + bh_kahan_smem_bytes<T>());
    auto kern = bh_walk_tma_kernel<T, ORDER>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return BH_ERR_CUDA;
    int bps = blocks_per_sm;
    if (bps <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, block_threads, smem) != cudaSuccess || bps < 1)
            bps = 1;
    }
    kern<<<sm_count * bps, block_threads, smem, s>>>(P);
    return BH_OK;
}

static int bh_walk_tma_dispatch(const WalkParams& P, int order, int G, int sm_count, int block_threads,
                                int blocks_per_sm, cudaStream_t s)
{
    const int T = G <= 32 ? 1 : G <= 64 ? 2 : G <= 96 ? 3 : G <= 128 ? 4 : 8;
    if (order >= 2) {
        switch (T) {
            case 1: return bh_walk_tma_launch_t<1, 2>(P, sm_count, block_threads, blocks_per_sm, s);
            case 2: return bh_walk_tma_launch_t<2, 2>(P, sm_count, block_threads, blocks_per_sm, s);
            case 3: return bh_walk_tma_launch_t<3, 2>(P, sm_count, block_threads, blocks_per_sm, s);
            case 4: return bh_walk_tma_launch_t<4, 2>(P, sm_count, block_threads, blocks_per_sm, s);
            default: return bh_walk_tma_launch_t<8, 2>(P, sm_count, block_threads, blocks_per_sm, s);
        }
    }
    switch (T) {
        case 1: return bh_walk_tma_launch_t<1, 1>(P, sm_count, block_threads, blocks_per_sm, s);
        case 2: return bh_walk_tma_launch_t<2, 1>(P, sm_count, block_threads, blocks_per_sm, s);
        case 3: return bh_walk_tma_launch_t<3, 1>(P, sm_count, block_threads, blocks_per_sm, s);
        case 4: return bh_walk_tma_launch_t<4, 1>(P, sm_count, block_threads, blocks_per_sm, s);
        default: return bh_walk_tma_launch_t<8, 1>(P, sm_count, block_threads, blocks_per_sm, s);
    }
}

// Self-test of the failure path: one warp waits on a tile-ring mbarrier that
// nothing will arrive on.  bh_mbar_wait gives up within a second and
// records BH_ERR_DEVICE_TIMEOUT, as a stalled pair of the paired walk would.
__global__ void bh_selftest_ring_kernel(bh_dev_ctrl* c)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) bh_mbar_init(&bar, 32u);
    __syncthreads();
    bh_mbar_wait(&bar, 0u, c);
}

void launch_selftest_ring(bh_dev_ctrl* c, cudaStream_t s)
{
    bh_selftest_ring_kernel<<<1, 32, 0, s>>>(c);
}

// Self-test of the TMA-staged walk's wait: the mbarrier is told to expect 16
// bytes (as a batch of copies would) but no copy is issued, so
// bh_mbar_wait_own gives up within a second and records BH_ERR_DEVICE_TIMEOUT.
// Nothing is in flight when the kernel returns.
__global__ void bh_selftest_tma_kernel(bh_dev_ctrl* c)
{
    __shared__ unsigned long long bar;
    if (threadIdx.x == 0) {
        bh_mbar_init(&bar, 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x == 0) bh_mbar_expect_tx(&bar, 16u);
    __syncwarp();
    bh_mbar_wait_own(&bar, 0u, c);
}

void launch_selftest_tma(bh_dev_ctrl* c, cudaStream_t s)
{
    bh_selftest_tma_kernel<<<1, 32, 0, s>>>(c);
}

__global__ void bh_walk_reset_kernel(bh_dev_ctrl* c)
{
    c->group_ctr = 0u;
    c->n_pp = 0ull;
    c->n_pc = 0ull;
}

template <int T, int ORDER, bool LEARNED>
static int bh_walk_launch_t(const WalkParams& P, int sm_count, int block_threads, int blocks_per_sm,
                            cudaStream_t s)
{
    const int nw = block_threads / 32;
    size_t smem = (size_t)nw * (sizeof(WarpSmem) + (ORDER >= 2 ? sizeof(WarpQuad) : 0));
    if (LEARNED) smem += sizeof(bh_mlp_dev) + (size_t)nw * 32 * 8 * sizeof(uint32_t);
    smem += (size_t)nw * bh_kahan_smem_bytes<T>();
    auto kern = bh_walk_kernel<T, ORDER, LEARNED>;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return BH_ERR_CUDA;
    }
    int bps = blocks_per_sm;
    if (bps <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, block_threads, smem) != cudaSuccess || bps < 1)
            bps = 1;
    }
    kern<<<sm_count * bps, block_threads, smem, s>>>(P);
    return BH_OK;
}

template <bool LEARNED>
static int bh_walk_dispatch(const WalkParams& P, int order, int G, int sm_count, int block_threads,
                            int blocks_per_sm, cudaStream_t s)
{
    // target slots per lane: ceil(G / 32), one instantiation per value up to 4
    const int T = G <= 32 ? 1 : G <= 64 ? 2 : G <= 96 ? 3 : G <= 128 ? 4 : 8;
    if (order >= 2) {
        switch (T) {
            case 1: return bh_walk_launch_t<1, 2, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
            case 2: return bh_walk_launch_t<2, 2, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
            case 3: return bh_walk_launch_t<3, 2, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
            case 4: return bh_walk_launch_t<4, 2, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
            default: return bh_walk_launch_t<8, 2, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
        }
    }
    switch (T) {
        case 1: return bh_walk_launch_t<1, 1, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
        case 2: return bh_walk_launch_t<2, 1, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
        case 3: return bh_walk_launch_t<3, 1, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
        case 4: return bh_walk_launch_t<4, 1, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
        default: return bh_walk_launch_t<8, 1, LEARNED>(P, sm_count, block_threads, blocks_per_sm, s);
    }
}

int launch_walk(const float4* pos_s, const uint32_t* perm, const int32_t* g_first, const int32_t* g_count,
                const bh_nodes& nd, int order, int G, float eps, float4* out, bh_dev_ctrl* ctrl, int sm_count,
                int block_threads, int blocks_per_sm, cudaStream_t s, const WalkLearned* learned, int walk_variant)
{
    bh_walk_reset_kernel<<<1, 1, 0, s>>>(ctrl);
    WalkParams P;
    P.pos_s = pos_s;
    P.perm = perm;
    P.g_first = g_first;
    P.g_count = g_count;
    P.rec = nd.rec;
    P.com_m = nd.com_m;
    P.seff = nd.seff;
    P.quad = nd.quad;
    P.out = out;
    P.ctrl = ctrl;
    P.eps2 = eps * eps;
    P.mfeat = nullptr;
    P.mlp = nullptr;
    P.theta_guard = 1.0f;
    P.wrec = nd.wrec;
    if (learned) {
        P.mfeat = learned->mfeat;
        P.mlp = learned->mlp;
        P.theta_guard = learned->theta_guard;
        return bh_walk_dispatch<true>(P, order, G, sm_count, block_threads, blocks_per_sm, s);
    }
    if (walk_variant == BH_WALK_TMA && nd.wrec)
        return bh_walk_tma_dispatch(P, order, G, sm_count, block_threads, blocks_per_sm, s);
    if (walk_variant == BH_WALK_PAIRED && G <= 96) {
        const int T = G <= 32 ? 1 : G <= 64 ? 2 : 3;
        if (order >= 2) {
            switch (T) {
                case 1: return bh_walk_ws_launch<1, 2>(P, sm_count, s);
                case 2: return bh_walk_ws_launch<2, 2>(P, sm_count, s);
                default: return bh_walk_ws_launch<3, 2>(P, sm_count, s);
            }
        }
        switch (T) {
            case 1: return bh_walk_ws_launch<1, 1>(P, sm_count, s);
            case 2: return bh_walk_ws_launch<2, 1>(P, sm_count, s);
            default: return bh_walk_ws_launch<3, 1>(P, sm_count, s);
        }
    }
    return bh_walk_dispatch<false>(P, order, G, sm_count, block_threads, blocks_per_sm, s);
}

}  // namespace bh

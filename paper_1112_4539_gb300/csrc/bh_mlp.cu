// bh_mlp.cu -- training and labelling kernels of the learned opening criterion.
//
// The criterion (an extension of Eq. 2's test) is trained on errors the method
// measures itself: for sampled groups the labelling kernel walks the tree
// with a permissive Eq. (2) guard and, for every node passing it, compares the
// node's particle-cell term with the direct sum over the node's particles on
// every group member, relative to the member's total acceleration.  The
// network is then fit by hand-written forward/backward kernels and Adam
// (Kingma & Ba 2015) on FP32 master weights.
#include <cmath>
#include <cstring>
#include <algorithm>

#include "bh_mlp.cuh"

namespace bh {

// ------------------------------------------------------------ features
__device__ __forceinline__ float bh_quad_aniso(const float4& q0, const float4& q1, float M, float side)
{
    // |I - (T/3) 1|_F / (M l^2) from (xx, yy, zz, xy), (xz, yz, 1.5T, 0.5T)
    const float T3 = (q0.x + q0.y + q0.z) * (1.0f / 3.0f);
    const float a = q0.x - T3, b = q0.y - T3, c = q0.z - T3;
    const float fro = sqrtf(a * a + b * b + c * c + 2.0f * (q0.w * q0.w + q1.x * q1.x + q1.y * q1.y));
    return (M > 0.f) ? fro / (M * side * side) : 0.f;
}

// Per node: (log10 M/M_tot, quadrupole anisotropy, level, log2(count)/24).
__global__ void __launch_bounds__(256) bh_mac_nodefeat_kernel(bh_nodes nd, int order, float4* __restrict__ mfeat,
                                                              const bh_dev_ctrl* __restrict__ c)
{
    const int nn = (int)c->n_nodes;
    if (nn == 0) return;
    const float mtot = nd.com_m[0].w, L = c->box[3];
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nn; v += gridDim.x * blockDim.x) {
        const float M = nd.com_m[v].w;
        const int lev = nd.level[v];
        const float side = ldexpf(L, -lev);
        float qa = 0.f;
        if (order >= 2) qa = bh_quad_aniso(nd.quad[2 * (size_t)v], nd.quad[2 * (size_t)v + 1], M, side);
        const float f2 = (M > 0.f && mtot > 0.f) ? log10f(M / mtot) : -30.0f;
        mfeat[v] = make_float4(f2, qa, (float)lev, log2f((float)nd.count[v]) * (1.0f / 24.0f));
    }
}

void launch_mac_nodefeat(const bh_nodes& nd, int order, float4* mfeat, bh_dev_ctrl* ctrl, int grid, cudaStream_t s)
{
    bh_mac_nodefeat_kernel<<<grid, 256, 0, s>>>(nd, order, mfeat, ctrl);
}

// ------------------------------------------------------------ labels
constexpr int kLabelWarps = 4;
constexpr int kLabelStack = 160;  // DFS: <= 7 pending siblings on each of 21 levels, + 8
constexpr int kLabelSlots = 8;    // members per lane (groups of up to 256)

struct LabelArgs {
    const float4* pos_s;
    const uint32_t* perm;
    const int32_t* g_first;
    const int32_t* g_count;
    const int32_t* groups;
    int n_groups;
    const int4* rec;
    const float4* com_m;
    const float* seff;
    const float4* quad;
    const float4* mfeat;
    const float4* acc_ref;
    float eps2;
    float log_floor;
    int order;
    float* X;
    float* Y;
    int32_t* pairs;
    long long cap;
    unsigned long long* count;
    bh_dev_ctrl* ctrl;
};

__global__ void __launch_bounds__(kLabelWarps * 32) bh_mac_label_kernel(LabelArgs A)
{
    __shared__ int s_stack[kLabelWarps][kLabelStack];
    __shared__ float4 s_tile[kLabelWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = blockIdx.x * kLabelWarps + w;
    if (gw >= A.n_groups) return;
    const int g = A.groups[gw];
    if (g < 0 || g >= (int)A.ctrl->n_groups) return;
    const int gb = A.g_first[g], gc = A.g_count[g], ge = gb + gc;
    if (gc > 32 * kLabelSlots) return;
    const float L = A.ctrl->box[3];
    float xi[kLabelSlots], yi[kLabelSlots], zi[kLabelSlots], at[kLabelSlots];
    float lo0 = INFINITY, lo1 = INFINITY, lo2 = INFINITY, hi0 = -INFINITY, hi1 = -INFINITY, hi2 = -INFINITY;
#pragma unroll
    for (int k = 0; k < kLabelSlots; k++) {
        const int o = k * 32 + lane;
        xi[k] = yi[k] = zi[k] = 0.f;
        at[k] = 1.f;
        if (o < gc) {
            const float4 p = A.pos_s[gb + o];
            xi[k] = p.x; yi[k] = p.y; zi[k] = p.z;
            const float4 a = A.acc_ref[A.perm[gb + o]];
            at[k] = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
            lo0 = fminf(lo0, p.x); lo1 = fminf(lo1, p.y); lo2 = fminf(lo2, p.z);
            hi0 = fmaxf(hi0, p.x); hi1 = fmaxf(hi1, p.y); hi2 = fmaxf(hi2, p.z);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo0 = fminf(lo0, __shfl_xor_sync(BH_FULL_MASK, lo0, o));
        lo1 = fminf(lo1, __shfl_xor_sync(BH_FULL_MASK, lo1, o));
        lo2 = fminf(lo2, __shfl_xor_sync(BH_FULL_MASK, lo2, o));
        hi0 = fmaxf(hi0, __shfl_xor_sync(BH_FULL_MASK, hi0, o));
        hi1 = fmaxf(hi1, __shfl_xor_sync(BH_FULL_MASK, hi1, o));
        hi2 = fmaxf(hi2, __shfl_xor_sync(BH_FULL_MASK, hi2, o));
    }
    const float gcx = 0.5f * (lo0 + hi0), gcy = 0.5f * (lo1 + hi1), gcz = 0.5f * (lo2 + hi2);
    const float rg = 0.5f * sqrtf((hi0 - lo0) * (hi0 - lo0) + (hi1 - lo1) * (hi1 - lo1) + (hi2 - lo2) * (hi2 - lo2));
    int* stack = s_stack[w];
    int sp = 1;
    if (lane == 0) stack[0] = 0;
    __syncwarp();
    while (sp > 0) {
        const int v = stack[sp - 1];
        sp--;
        __syncwarp();
        const int4 r = A.rec[v];
        const float4 cm = A.com_m[v];
        const float dx = fmaxf(fmaxf(lo0 - cm.x, cm.x - hi0), 0.f);
        const float dy = fmaxf(fmaxf(lo1 - cm.y, cm.y - hi1), 0.f);
        const float dz = fmaxf(fmaxf(lo2 - cm.z, cm.z - hi2), 0.f);
        const bool member = (r.x < ge) && (r.x + r.y > gb);
        const bool guard = !member && (dx * dx + dy * dy + dz * dz > A.seff[v]);
        bool descend = !guard;
        if (guard) {
            float f[BH_MLP_NF], side;
            const bool ok = bh_mac_features(cm, A.mfeat[v], gcx, gcy, gcz, rg, L, f, side);
            float4 q0 = make_float4(0.f, 0.f, 0.f, 0.f), q1 = q0;
            if (A.order >= 2) {
                q0 = A.quad[2 * (size_t)v];
                q1 = A.quad[2 * (size_t)v + 1];
            }
            // particle-cell term on every member
            float px[kLabelSlots], py[kLabelSlots], pz[kLabelSlots];
#pragma unroll
            for (int k = 0; k < kLabelSlots; k++) {
                const float rx = xi[k] - cm.x, ry = yi[k] - cm.y, rz = zi[k] - cm.z;
                const float h2 = rx * rx + ry * ry + rz * rz + A.eps2;
                const float g1 = rsqrtf(h2), g2 = g1 * g1, g3 = g1 * g2, g5 = g3 * g2, g7 = g5 * g2;
                const float ir0 = q0.x * rx + q0.w * ry + q1.x * rz;
                const float ir1 = q0.w * rx + q0.y * ry + q1.y * rz;
                const float ir2 = q1.x * rx + q1.y * ry + q0.z * rz;
                const float q = rx * ir0 + ry * ir1 + rz * ir2;
                const float kk = q1.z * g5 - 7.5f * q * g7 - cm.w * g3;
                px[k] = kk * rx + 3.f * g5 * ir0;
                py[k] = kk * ry + 3.f * g5 * ir1;
                pz[k] = kk * rz + 3.f * g5 * ir2;
            }
            // exact sum over the node's particles (FP32 tiles, Kahan across tiles)
            float ex[kLabelSlots], ey[kLabelSlots], ez[kLabelSlots], cx[kLabelSlots], cy[kLabelSlots],
                cz[kLabelSlots];
#pragma unroll
            for (int k = 0; k < kLabelSlots; k++) ex[k] = ey[k] = ez[k] = cx[k] = cy[k] = cz[k] = 0.f;
            for (int j0 = r.x; j0 < r.x + r.y; j0 += 32) {
                const int jn = min(32, r.x + r.y - j0);
                s_tile[w][lane] = (lane < jn) ? A.pos_s[j0 + lane] : make_float4(1e18f, 1e18f, 1e18f, 0.f);
                __syncwarp();
#pragma unroll
                for (int k = 0; k < kLabelSlots; k++) {
                    if (k * 32 >= gc) break;
                    float tx = 0.f, ty = 0.f, tz = 0.f;
                    for (int j = 0; j < 32; j++) {
                        const float4 s = s_tile[w][j];
                        const float ddx = s.x - xi[k], ddy = s.y - yi[k], ddz = s.z - zi[k];
                        const float r2 = ddx * ddx + ddy * ddy + ddz * ddz + A.eps2;
                        const float ri = rsqrtf(r2);
                        const float mr3 = s.w * ri * ri * ri;
                        tx = fmaf(mr3, ddx, tx);
                        ty = fmaf(mr3, ddy, ty);
                        tz = fmaf(mr3, ddz, tz);
                    }
                    float yv = tx - cx[k], tv = ex[k] + yv;
                    cx[k] = (tv - ex[k]) - yv; ex[k] = tv;
                    yv = ty - cy[k]; tv = ey[k] + yv;
                    cy[k] = (tv - ey[k]) - yv; ey[k] = tv;
                    yv = tz - cz[k]; tv = ez[k] + yv;
                    cz[k] = (tv - ez[k]) - yv; ez[k] = tv;
                }
                __syncwarp();
            }
            float worst = 0.f;
#pragma unroll
            for (int k = 0; k < kLabelSlots; k++) {
                if (k * 32 + lane < gc) {
                    const float ddx = px[k] - (ex[k] - cx[k]), ddy = py[k] - (ey[k] - cy[k]),
                                ddz = pz[k] - (ez[k] - cz[k]);
                    worst = fmaxf(worst, sqrtf(ddx * ddx + ddy * ddy + ddz * ddz) / at[k]);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(BH_FULL_MASK, worst, o));
            const float label = log10f(fmaxf(worst, 1e-12f));
            if (ok && lane == 0) {
                const unsigned long long idx = atomicAdd(A.count, 1ull);
                if ((long long)idx < A.cap) {
                    for (int k = 0; k < BH_MLP_NF; k++) A.X[idx * BH_MLP_NF + k] = f[k];
                    A.Y[idx] = label;
                    if (A.pairs) {
                        A.pairs[2 * idx] = v;
                        A.pairs[2 * idx + 1] = g;
                    }
                }
            }
            descend = label > A.log_floor;
        }
        if (descend && r.z >= 0) {
            if (sp + r.w > kLabelStack) {
                if (lane == 0) bh_set_error(A.ctrl, BH_ERR_CAPACITY);
                return;
            }
            if (lane < r.w) stack[sp + r.w - 1 - lane] = r.z + lane;
            sp += r.w;
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------ training
// Activation record per sample: x[6], pre1 mask via h1 > 0, h1[32], h2[32],
// d1[32] (loss gradient at layer-1 pre-activation), d2[32], dy.
constexpr int kAct = BH_MLP_NF + 4 * BH_MLP_NH + 1;
constexpr int kOffB1 = BH_MLP_NH * BH_MLP_NF, kOffW2 = kOffB1 + BH_MLP_NH, kOffB2 = kOffW2 + BH_MLP_NH * BH_MLP_NH,
              kOffW3 = kOffB2 + BH_MLP_NH, kOffB3 = kOffW3 + BH_MLP_NH;

__global__ void __launch_bounds__(256) bh_mlp_fwd_bwd_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                             const float* __restrict__ Y,
                                                             const int32_t* __restrict__ order, long long i0, int B,
                                                             long long n, float under_w, float* __restrict__ act,
                                                             float* __restrict__ loss, float* __restrict__ yhat)
{
    __shared__ float sp[BH_MLP_NPARAM];
    for (int i = threadIdx.x; i < BH_MLP_NPARAM; i += blockDim.x) sp[i] = P[i];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const long long s = order ? (long long)order[(i0 + b) % n] : (i0 + b) % n;
    float x[BH_MLP_NF], h1[BH_MLP_NH], h2[BH_MLP_NH];
    for (int k = 0; k < BH_MLP_NF; k++) x[k] = X[s * BH_MLP_NF + k];
    for (int j = 0; j < BH_MLP_NH; j++) {
        float a = sp[kOffB1 + j];
        for (int k = 0; k < BH_MLP_NF; k++) a = fmaf(sp[j * BH_MLP_NF + k], x[k], a);
        h1[j] = fmaxf(a, 0.f);
    }
    for (int j = 0; j < BH_MLP_NH; j++) {
        float a = sp[kOffB2 + j];
        for (int k = 0; k < BH_MLP_NH; k++) a = fmaf(sp[kOffW2 + j * BH_MLP_NH + k], h1[k], a);
        h2[j] = fmaxf(a, 0.f);
    }
    float y = sp[kOffB3];
    for (int k = 0; k < BH_MLP_NH; k++) y = fmaf(sp[kOffW3 + k], h2[k], y);
    if (yhat) yhat[b] = y;
    if (!act) return;
    const float t = Y[s], r = y - t, wgt = (y < t) ? under_w : 1.0f;
    if (loss) atomicAdd(loss, wgt * r * r / (float)B);
    const float dy = 2.0f * wgt * r / (float)B;
    float* a = act + (size_t)b * kAct;
    for (int k = 0; k < BH_MLP_NF; k++) a[k] = x[k];
    float d2[BH_MLP_NH];
    for (int k = 0; k < BH_MLP_NH; k++) {
        a[BH_MLP_NF + k] = h1[k];
        a[BH_MLP_NF + BH_MLP_NH + k] = h2[k];
        d2[k] = h2[k] > 0.f ? dy * sp[kOffW3 + k] : 0.f;
        a[BH_MLP_NF + 3 * BH_MLP_NH + k] = d2[k];
    }
    for (int k = 0; k < BH_MLP_NH; k++) {
        float d = 0.f;
        for (int j = 0; j < BH_MLP_NH; j++) d = fmaf(d2[j], sp[kOffW2 + j * BH_MLP_NH + k], d);
        a[BH_MLP_NF + 2 * BH_MLP_NH + k] = h1[k] > 0.f ? d : 0.f;
    }
    a[kAct - 1] = dy;
}

// Gradient of the mean loss: block j < 32 reduces hidden unit j's rows of
// W1, b1, W2, b2 over the batch; block 32 reduces W3 and b3.
__global__ void __launch_bounds__(256) bh_mlp_grad_kernel(const float* __restrict__ act, int B,
                                                          float* __restrict__ grad)
{
    constexpr int kOut = BH_MLP_NF + 1 + BH_MLP_NH + 1;  // 40 accumulators per thread
    __shared__ float red[kOut][33];
    const int j = blockIdx.x;
    float acc[kOut];
#pragma unroll
    for (int k = 0; k < kOut; k++) acc[k] = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float* a = act + (size_t)b * kAct;
        if (j < BH_MLP_NH) {
            const float d1 = a[BH_MLP_NF + 2 * BH_MLP_NH + j], d2 = a[BH_MLP_NF + 3 * BH_MLP_NH + j];
#pragma unroll
            for (int k = 0; k < BH_MLP_NF; k++) acc[k] = fmaf(d1, a[k], acc[k]);
            acc[BH_MLP_NF] += d1;
#pragma unroll
            for (int k = 0; k < BH_MLP_NH; k++) acc[BH_MLP_NF + 1 + k] = fmaf(d2, a[BH_MLP_NF + k], acc[BH_MLP_NF + 1 + k]);
            acc[kOut - 1] += d2;
        } else {
            const float dy = a[kAct - 1];
#pragma unroll
            for (int k = 0; k < BH_MLP_NH; k++) acc[k] = fmaf(dy, a[BH_MLP_NF + BH_MLP_NH + k], acc[k]);
            acc[BH_MLP_NH] += dy;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kOut; k++) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(BH_FULL_MASK, v, o);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kOut) {
        float v = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) v += red[threadIdx.x][i];
        const int k = threadIdx.x;
        if (j < BH_MLP_NH) {
            if (k < BH_MLP_NF) grad[j * BH_MLP_NF + k] = v;
            else if (k == BH_MLP_NF) grad[kOffB1 + j] = v;
            else if (k < kOut - 1) grad[kOffW2 + j * BH_MLP_NH + (k - BH_MLP_NF - 1)] = v;
            else grad[kOffB2 + j] = v;
        } else {
            if (k < BH_MLP_NH) grad[kOffW3 + k] = v;
            else if (k == BH_MLP_NH) grad[kOffB3] = v;
        }
    }
}

__global__ void bh_adam_kernel(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                               float* __restrict__ v, long long t, float lr, float b1, float b2, float eps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= BH_MLP_NPARAM) return;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    const float mk = b1 * m[k] + (1.f - b1) * g[k];
    const float vk = b2 * v[k] + (1.f - b2) * g[k] * g[k];
    m[k] = mk;
    v[k] = vk;
    P[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Inference path: the walk's tensor-core network, 32 samples per warp.
__global__ void __launch_bounds__(128) bh_mlp_mma_forward_kernel(const bh_mlp_dev* __restrict__ Wg,
                                                                 const float* __restrict__ X, long long n,
                                                                 float* __restrict__ y)
{
    __shared__ bh_mlp_dev W;
    __shared__ uint32_t xs[4][32 * 8];
    for (int i = threadIdx.x; i < (int)(sizeof(bh_mlp_dev) / 4); i += blockDim.x)
        reinterpret_cast<uint32_t*>(&W)[i] = reinterpret_cast<const uint32_t*>(Wg)[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long s = ((long long)blockIdx.x * 4 + w) * 32 + lane;
    float f[BH_MLP_NF];
    for (int k = 0; k < BH_MLP_NF; k++) f[k] = (s < n) ? X[s * BH_MLP_NF + k] : 0.f;
    const float v = bh_mlp_warp(W, xs[w], f);
    if (s < n) y[s] = v;
}

// ------------------------------------------------------------ host side
static uint16_t bf16_bits(float x)
{
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    uint16_t u;
    std::memcpy(&u, &b, 2);
    return u;
}

void mlp_pack(const float* P, const float* fmin, const float* fmax, float ltau, float theta_fb, bh_mlp_dev* out)
{
    std::memset(out, 0, sizeof(*out));
    auto pack = [](float lo, float hi) { return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16); };
    // word w of a row of K = 32 holds k = 2w, 2w + 1; k-step s, lane t of the
    // quad takes words 8s + t and 8s + t + 4
    auto word32 = [&](int off, int w) { return pack(P[off + 2 * w], P[off + 2 * w + 1]); };
    for (int j = 0; j < 32; j++) {
        for (int w = 0; w < 4; w++) {
            const int k0 = 2 * w, k1 = 2 * w + 1;
            out->w1[j][w] = pack(k0 < BH_MLP_NF ? P[j * BH_MLP_NF + k0] : 0.f, k1 < BH_MLP_NF ? P[j * BH_MLP_NF + k1] : 0.f);
        }
        for (int ks = 0; ks < 2; ks++)
            for (int t = 0; t < 4; t++)
                out->w2[j][ks][t] = make_uint2(word32(kOffW2 + j * 32, 8 * ks + t), word32(kOffW2 + j * 32, 8 * ks + t + 4));
        out->b1[j] = P[kOffB1 + j];
        out->b2[j] = P[kOffB2 + j];
    }
    for (int ks = 0; ks < 2; ks++)
        for (int t = 0; t < 4; t++)
            out->w3[0][ks][t] = make_uint2(word32(kOffW3, 8 * ks + t), word32(kOffW3, 8 * ks + t + 4));
    out->b3[0] = P[kOffB3];
    for (int k = 0; k < 8; k++) {
        out->fmin[k] = k < BH_MLP_NF ? fmin[k] : -INFINITY;
        out->fmax[k] = k < BH_MLP_NF ? fmax[k] : INFINITY;
    }
    out->ltau = ltau;
    out->theta_fb = theta_fb;
}

int mac_label(const float4* pos_s, const uint32_t* perm, const int32_t* g_first, const int32_t* g_count,
              const int32_t* groups, int n_groups, const bh_nodes& nd, const float4* mfeat, const float4* acc_ref,
              float eps, float log_floor, int order, float* X, float* Y, int32_t* pairs, long long cap,
              unsigned long long* count, bh_dev_ctrl* ctrl, cudaStream_t s)
{
    if (n_groups <= 0) return BH_OK;
    LabelArgs a;
    a.pairs = pairs;
    a.pos_s = pos_s;
    a.perm = perm;
    a.g_first = g_first;
    a.g_count = g_count;
    a.groups = groups;
    a.n_groups = n_groups;
    a.rec = nd.rec;
    a.com_m = nd.com_m;
    a.seff = nd.seff;
    a.quad = nd.quad;
    a.mfeat = mfeat;
    a.acc_ref = acc_ref;
    a.eps2 = eps * eps;
    a.log_floor = log_floor;
    a.order = order;
    a.X = X;
    a.Y = Y;
    a.cap = cap;
    a.count = count;
    a.ctrl = ctrl;
    bh_mac_label_kernel<<<(n_groups + kLabelWarps - 1) / kLabelWarps, kLabelWarps * 32, 0, s>>>(a);
    return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

int mlp_train(const float* X, const float* Y, const int32_t* order, long long n, float* P, float* adam_m,
              float* adam_v, float* work, long long work_floats, long long steps, int batch, float lr,
              float under_w, float* loss, long long t0, cudaStream_t s)
{
    if (batch < 1 || n < 1 || steps < 0) return BH_ERR_INVALID;
    const long long need = (long long)batch * kAct + BH_MLP_NPARAM;
    if (work_floats < need) return BH_ERR_TOO_LARGE;
    float* act = work;
    float* grad = work + (size_t)batch * kAct;
    const int blocks = (batch + 255) / 256;
    for (long long st = 0; st < steps; st++) {
        const long long i0 = ((t0 + st) * (long long)batch) % n;
        bh_mlp_fwd_bwd_kernel<<<blocks, 256, 0, s>>>(P, X, Y, order, i0, batch, n, under_w, act,
                                                     loss ? loss + st : nullptr, nullptr);
        bh_mlp_grad_kernel<<<BH_MLP_NH + 1, 256, 0, s>>>(act, batch, grad);
        bh_adam_kernel<<<(BH_MLP_NPARAM + 255) / 256, 256, 0, s>>>(P, grad, adam_m, adam_v, t0 + st + 1, lr, 0.9f,
                                                                   0.999f, 1e-8f);
    }
    return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

int mlp_grad(const float* P, const float* X, const float* Y, long long n, float under_w, float* work,
             long long work_floats, float* grad, float* loss, cudaStream_t s)
{
    const long long need = n * kAct;
    if (work_floats < need) return BH_ERR_TOO_LARGE;
    if (n > (1ll << 30)) return BH_ERR_TOO_LARGE;
    bh_mlp_fwd_bwd_kernel<<<(int)((n + 255) / 256), 256, 0, s>>>(P, X, Y, nullptr, 0, (int)n, n, under_w, work, loss,
                                                                 nullptr);
    bh_mlp_grad_kernel<<<BH_MLP_NH + 1, 256, 0, s>>>(work, (int)n, grad);
    return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

int mlp_forward(const float* P, const bh_mlp_dev* Wdev, const float* X, long long n, float* y, int precision,
                cudaStream_t s)
{
    if (n <= 0) return BH_OK;
    if (precision == 16) {
        bh_mlp_mma_forward_kernel<<<(int)((n + 127) / 128), 128, 0, s>>>(Wdev, X, n, y);
    } else {
        // FP32 training forward, in chunks the kernel's int batch can index
        for (long long i0 = 0; i0 < n; i0 += (1ll << 30)) {
            const int B = (int)std::min<long long>(n - i0, 1ll << 30);
            bh_mlp_fwd_bwd_kernel<<<(B + 255) / 256, 256, 0, s>>>(P, X, nullptr, nullptr, i0, B, n, 1.f, nullptr,
                                                                  nullptr, y + i0);
        }
    }
    return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

}  // namespace bh

// bh_mlp.cuh -- the learned opening criterion's network on the device.
//
// The criterion extends Eq. (2)'s test: a 6 -> 32 -> 32 -> 1 ReLU network
// predicts log10 of a node's relative force-error contribution to a group of
// targets from six features (node side / distance, log10 mass fraction,
// quadrupole anisotropy, group radius / distance, depth, log2 count).  In the
// walk it runs on the tensor cores as one warp-wide BF16 contraction per
// batch of 32 tested nodes (mma.sync, FP32 accumulate): the 32 nodes are the
// M dimension, features / hidden units the K and N ones.  Layer 1 has K = 6
// (padded to 8: m16n8k8), layers 2 and 3 K = 32 (two m16n8k16 steps).
#pragma once

#include <cuda_bf16.h>

#include "bh_internal.cuh"

#define BH_MLP_NF 6
#define BH_MLP_NH 32
#define BH_MLP_NPARAM (BH_MLP_NH * BH_MLP_NF + BH_MLP_NH + BH_MLP_NH * BH_MLP_NH + BH_MLP_NH + BH_MLP_NH + 1)

// Inference parameters, BF16 weights packed as pairs along K, rows = output
// units, in B-fragment order: w1[n][t] holds k = 2t, 2t+1 of row n (the one
// register of m16n8k8); w2[n][s][t] and w3[n][s][t] hold the two registers of
// k-step s of m16n8k16 (k = 16s + 2t, 2t+1 and k = 16s + 8 + 2t, 2t+1), so
// each fragment is one shared-memory load.
struct __align__(16) bh_mlp_dev {
    uint32_t w1[32][4];   // layer 1: K = 6 features padded to 8
    uint2 w2[32][2][4];   // layer 2: K = 32
    uint2 w3[8][2][4];    // layer 3: only output row 0 is non-zero
    float b1[32];
    float b2[32];
    float b3[8];
    float fmin[8];        // training range of each feature; outside it the
    float fmax[8];        // plain criterion at theta_fb decides
    float ltau;           // log10(tau): accept when the prediction is below
    float theta_guard;    // theta of the guard's S_eff
    float theta_fb;
    float pad;
};

__device__ __forceinline__ uint32_t bh_pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// max(lo, 0), max(hi, 0) rounded to bfloat16 (nearest even) and packed as
// bh_pack_bf16 packs them: one conversion instruction with ReLU, which gives
// the same bits as rounding max(x, 0) for every finite x.
__device__ __forceinline__ uint32_t bh_pack_bf16_relu(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void bh_mma_bf16_k8(float (&d)[4], const uint32_t (&a)[2], uint32_t b0)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(b0));
}

__device__ __forceinline__ void bh_mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Network prediction for the sample held by each lane (features f[6]).
// W: parameters in shared memory; xs: this warp's staging area (32 x 4 words
// used; callers reserve 32 x 8).
// Must be called by all 32 lanes of the warp.
__device__ __forceinline__ float bh_mlp_warp(const bh_mlp_dev& W, uint32_t* xs, const float (&f)[BH_MLP_NF])
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // stage this lane's features as a row of 8 bf16 (words 0..2 real, 3 zero)
    xs[lane * 4 + 0] = bh_pack_bf16(f[0], f[1]);
    xs[lane * 4 + 1] = bh_pack_bf16(f[2], f[3]);
    xs[lane * 4 + 2] = bh_pack_bf16(f[4], f[5]);
    xs[lane * 4 + 3] = 0u;
    __syncwarp();
    float out[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
        const int r0 = mt * 16 + g, r1 = r0 + 8;
        const uint32_t a1[2] = {xs[r0 * 4 + t], xs[r1 * 4 + t]};
        // layer 1: 4 n-tiles of hidden units, bias in the accumulator
        float h1[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            const float2 b = reinterpret_cast<const float2*>(W.b1)[nt * 4 + t];  // b1[c], b1[c + 1], c = 8 nt + 2t
            h1[nt][0] = b.x;
            h1[nt][1] = b.y;
            h1[nt][2] = b.x;
            h1[nt][3] = b.y;
            bh_mma_bf16_k8(h1[nt], a1, W.w1[nt * 8 + g][t]);
        }
        // ReLU; the accumulators of n-tiles (2ks, 2ks+1) are the A fragment of k-step ks
        uint32_t a2[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            a2[ks][0] = bh_pack_bf16_relu(h1[2 * ks][0], h1[2 * ks][1]);
            a2[ks][1] = bh_pack_bf16_relu(h1[2 * ks][2], h1[2 * ks][3]);
            a2[ks][2] = bh_pack_bf16_relu(h1[2 * ks + 1][0], h1[2 * ks + 1][1]);
            a2[ks][3] = bh_pack_bf16_relu(h1[2 * ks + 1][2], h1[2 * ks + 1][3]);
        }
        float h2[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            const float2 b = reinterpret_cast<const float2*>(W.b2)[nt * 4 + t];
            h2[nt][0] = b.x;
            h2[nt][1] = b.y;
            h2[nt][2] = b.x;
            h2[nt][3] = b.y;
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                const uint2 w = W.w2[nt * 8 + g][ks][t];
                bh_mma_bf16(h2[nt], a2[ks], w.x, w.y);
            }
        }
        uint32_t a3[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            a3[ks][0] = bh_pack_bf16_relu(h2[2 * ks][0], h2[2 * ks][1]);
            a3[ks][1] = bh_pack_bf16_relu(h2[2 * ks][2], h2[2 * ks][3]);
            a3[ks][2] = bh_pack_bf16_relu(h2[2 * ks + 1][0], h2[2 * ks + 1][1]);
            a3[ks][3] = bh_pack_bf16_relu(h2[2 * ks + 1][2], h2[2 * ks + 1][3]);
        }
        float y[4] = {W.b3[2 * t], W.b3[2 * t + 1], W.b3[2 * t], W.b3[2 * t + 1]};
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            const uint2 w = W.w3[g][ks][t];
            bh_mma_bf16(y, a3[ks], w.x, w.y);
        }
        out[mt][0] = y[0];  // row r0, output column 2t (column 0 on lanes with t = 0)
        out[mt][1] = y[2];  // row r1
    }
    __syncwarp();
    // node `lane` sits in m-tile lane/16, row lane%16: held by lane 4*(lane%8)
    const int src = 4 * (lane & 7);
    const float v00 = __shfl_sync(BH_FULL_MASK, out[0][0], src);
    const float v01 = __shfl_sync(BH_FULL_MASK, out[0][1], src);
    const float v10 = __shfl_sync(BH_FULL_MASK, out[1][0], src);
    const float v11 = __shfl_sync(BH_FULL_MASK, out[1][1], src);
    const int rr = lane & 15;
    if (lane < 16) return rr < 8 ? v00 : v01;
    return rr < 8 ? v10 : v11;
}

// Features of (group, node), shared by the walk and the labelling kernel:
// nf = node-constant (log10 M/M_tot, quadrupole anisotropy, level, log2(count)/24),
// (gc, rg) = group box centre and half diagonal, L = root cube side.
__device__ __forceinline__ bool bh_mac_features(const float4& cm, const float4& nf, float gcx, float gcy, float gcz,
                                                float rg, float L, float (&f)[BH_MLP_NF], float& side)
{
    const int lev = (int)nf.z;
    side = ldexpf(L, -lev);
    const float ex = cm.x - gcx, ey = cm.y - gcy, ez = cm.z - gcz;
    const float dc = sqrtf(ex * ex + ey * ey + ez * ez);
    const float idc = dc > 0.f ? 1.0f / dc : 0.f;
    f[0] = side * idc;
    f[1] = nf.x;
    f[2] = nf.y;
    f[3] = rg * idc;
    f[4] = (float)lev * 0.1f;
    f[5] = nf.w;
    return dc > 0.f;
}


namespace bh {
struct LabelArgs;
void launch_mac_nodefeat(const bh_nodes& nd, int order, float4* mfeat, bh_dev_ctrl* ctrl, int grid, cudaStream_t s);
void mlp_pack(const float* P, const float* fmin, const float* fmax, float ltau, float theta_fb, bh_mlp_dev* out);
int mlp_train(const float* X, const float* Y, const int32_t* order, long long n, float* P, float* adam_m,
              float* adam_v, float* work, long long work_floats, long long steps, int batch, float lr,
              float under_w, float* loss, long long t0, cudaStream_t s);
int mlp_grad(const float* P, const float* X, const float* Y, long long n, float under_w, float* work,
             long long work_floats, float* grad, float* loss, cudaStream_t s);
int mlp_forward(const float* P, const bh_mlp_dev* Wdev, const float* X, long long n, float* y, int precision,
                cudaStream_t s);
int mac_label(const float4* pos_s, const uint32_t* perm, const int32_t* g_first, const int32_t* g_count,
              const int32_t* groups, int n_groups, const bh_nodes& nd, const float4* mfeat, const float4* acc_ref,
              float eps, float log_floor, int order, float* X, float* Y, int32_t* pairs, long long cap,
              unsigned long long* count, bh_dev_ctrl* ctrl, cudaStream_t s);
}  // namespace bh

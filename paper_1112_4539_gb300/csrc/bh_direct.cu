// bh_direct.cu -- Eq. (1) by direct summation (Sec. 3's brute-force method).
//
// One thread per target, sources staged through shared memory in tiles of
// 256.  FP32: rsqrtf interactions, plain sums within a tile, Kahan-compensated
// across tiles.  FP64: the error judge, double throughout with 1/sqrt.  When
// there are too few targets to fill the GPU the source range is split across
// blocks and partial sums are combined with atomic adds into the (zeroed)
// output.  The self term of each target is skipped by index.  With
// individual softening lengths (SYM) a pair softens with (eps_i^2 + eps_j^2)/2,
// the symmetrized Plummer potential (Sec. 7, after Saitoh & Makino 2010).
#include "bh_internal.cuh"

namespace bh {

constexpr int kDirThreads = 256;

template <typename R>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = bh_double4;
};

__device__ __forceinline__ float bh_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double bh_rsqrt(double x) { return 1.0 / sqrt(x); }

template <typename R>
__device__ __forceinline__ void bh_kahan_r(R& s, R& c, R v)
{
    const R y = v - c;
    const R t = s + y;  // no contraction or reassociation: adds only, no fast-math
    c = (t - s) - y;
    s = t;
}

template <typename R, bool ATOMIC, bool SYM = false>
__global__ void __launch_bounds__(kDirThreads)
bh_direct_kernel(const float4* __restrict__ src, int n_src, const float4* __restrict__ tgt,
                 const int64_t* __restrict__ self, int n_tgt, R eps2, typename Vec4<R>::type* __restrict__ out,
                 int chunk, const float* __restrict__ eps_src = nullptr, const float* __restrict__ eps_tgt = nullptr)
{
    __shared__ float4 tile[kDirThreads];
    __shared__ R tile_e[SYM ? kDirThreads : 1];  // eps_j^2 / 2
    const int i = blockIdx.x * kDirThreads + threadIdx.x;
    const bool valid = i < n_tgt;
    float4 pt = make_float4(0.f, 0.f, 0.f, 0.f);
    long long sf = -1;
    if (valid) {
        pt = tgt[i];
        if (self) sf = (long long)self[i];
    }
    const R xi = pt.x, yi = pt.y, zi = pt.z;
    R hi = 0;
    if (SYM && valid) {
        const R e = eps_tgt[i];
        hi = (R)0.5 * (e * e);
    }
    R ax = 0, ay = 0, az = 0, ph = 0, cx = 0, cy = 0, cz = 0, cp = 0;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(n_src, s0 + chunk);
    for (int base = s0; base < s1; base += kDirThreads) {
        const int j = base + threadIdx.x;
        tile[threadIdx.x] = (j < s1) ? src[j] : make_float4(1e18f, 1e18f, 1e18f, 0.0f);
        if (SYM) {
            const R e = (j < s1) ? (R)eps_src[j] : (R)0;
            tile_e[threadIdx.x] = (R)0.5 * (e * e);
        }
        __syncthreads();
        R tx = 0, ty = 0, tz = 0, tp = 0;
        const bool mine = sf >= base && sf < base + kDirThreads;
        const int skip = mine ? (int)(sf - base) : -1;
#pragma unroll 8
        for (int k = 0; k < kDirThreads; k++) {
            const float4 s = tile[k];
            const R dx = (R)s.x - xi, dy = (R)s.y - yi, dz = (R)s.z - zi;
            R r2 = dx * dx + dy * dy + dz * dz + (SYM ? hi + tile_e[k] : eps2);
            R m = s.w;
            if (k == skip) {
                r2 = 1;
                m = 0;
            }
            const R ri = bh_rsqrt(r2);
            const R mr = m * ri;
            const R mr3 = mr * ri * ri;
            tx += mr3 * dx;
            ty += mr3 * dy;
            tz += mr3 * dz;
            tp -= mr;
        }
        bh_kahan_r<R>(ax, cx, tx);
        bh_kahan_r<R>(ay, cy, ty);
        bh_kahan_r<R>(az, cz, tz);
        bh_kahan_r<R>(ph, cp, tp);
        __syncthreads();
    }
    if (!valid) return;
    const R rx = ax - cx, ry = ay - cy, rz = az - cz, rp = ph - cp;
    if (ATOMIC) {
        R* o = reinterpret_cast<R*>(out + i);
        atomicAdd(o + 0, rx);
        atomicAdd(o + 1, ry);
        atomicAdd(o + 2, rz);
        atomicAdd(o + 3, rp);
    } else {
        typename Vec4<R>::type v;
        v.x = rx;
        v.y = ry;
        v.z = rz;
        v.w = rp;
        out[i] = v;
    }
}

int launch_direct(const float4* src, int n_src, const float4* tgt, const int64_t* self, int n_tgt, double eps,
                  void* out, int precision, cudaStream_t s, const float* eps_src, const float* eps_tgt)
{
    const bool sym = eps_src != nullptr;
    if (n_tgt <= 0) return BH_OK;
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tblocks = (n_tgt + kDirThreads - 1) / kDirThreads;
    // split the sources when the targets alone give under ~8 blocks per SM
    int split = 1;
    if (tblocks < 8 * sms && n_src > 4 * kDirThreads) {
        split = (8 * sms + tblocks - 1) / tblocks;
        split = min(split, (n_src + 4 * kDirThreads - 1) / (4 * kDirThreads));
        split = max(split, 1);
    }
    const int chunk = ((n_src + split - 1) / split + kDirThreads - 1) / kDirThreads * kDirThreads;
    split = max(1, (n_src + chunk - 1) / max(chunk, 1));
    const dim3 grid(tblocks, split);
    const size_t rec = precision == 64 ? sizeof(bh_double4) : sizeof(float4);
    if (split > 1 || n_src == 0) cudaMemsetAsync(out, 0, (size_t)n_tgt * rec, s);
    if (n_src == 0) return BH_OK;
    if (sym) {
        if (precision == 64) {
            if (split > 1)
                bh_direct_kernel<double, true, true><<<grid, kDirThreads, 0, s>>>(
                    src, n_src, tgt, self, n_tgt, 0.0, (bh_double4*)out, chunk, eps_src, eps_tgt);
            else
                bh_direct_kernel<double, false, true><<<grid, kDirThreads, 0, s>>>(
                    src, n_src, tgt, self, n_tgt, 0.0, (bh_double4*)out, chunk, eps_src, eps_tgt);
        } else {
            if (split > 1)
                bh_direct_kernel<float, true, true><<<grid, kDirThreads, 0, s>>>(
                    src, n_src, tgt, self, n_tgt, 0.0f, (float4*)out, chunk, eps_src, eps_tgt);
            else
                bh_direct_kernel<float, false, true><<<grid, kDirThreads, 0, s>>>(
                    src, n_src, tgt, self, n_tgt, 0.0f, (float4*)out, chunk, eps_src, eps_tgt);
        }
    } else if (precision == 64) {
        if (split > 1)
            bh_direct_kernel<double, true><<<grid, kDirThreads, 0, s>>>(src, n_src, tgt, self, n_tgt, eps * eps,
                                                                        (bh_double4*)out, chunk);
        else
            bh_direct_kernel<double, false><<<grid, kDirThreads, 0, s>>>(src, n_src, tgt, self, n_tgt, eps * eps,
                                                                         (bh_double4*)out, chunk);
    } else {
        const float e2 = (float)(eps * eps);
        if (split > 1)
            bh_direct_kernel<float, true><<<grid, kDirThreads, 0, s>>>(src, n_src, tgt, self, n_tgt, e2,
                                                                       (float4*)out, chunk);
        else
            bh_direct_kernel<float, false><<<grid, kDirThreads, 0, s>>>(src, n_src, tgt, self, n_tgt, e2,
                                                                        (float4*)out, chunk);
    }
    return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

}  // namespace bh

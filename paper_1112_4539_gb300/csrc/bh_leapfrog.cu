// bh_leapfrog.cu -- the orbit-integration step around the force evaluation
// (Sec. 1: compute the forces, integrate the orbits, repeat).
#include "bh_internal.cuh"

namespace bh {

__global__ void __launch_bounds__(256) bh_kick_drift_kernel(float4* __restrict__ pos, float4* __restrict__ vel,
                                                            const float4* __restrict__ acc, int n, float dt_kick,
                                                            float dt_drift)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 a = acc[i];
        float4 v = vel[i];
        float4 x = pos[i];
        v.x = fmaf(a.x, dt_kick, v.x);
        v.y = fmaf(a.y, dt_kick, v.y);
        v.z = fmaf(a.z, dt_kick, v.z);
        x.x = fmaf(v.x, dt_drift, x.x);
        x.y = fmaf(v.y, dt_drift, x.y);
        x.z = fmaf(v.z, dt_drift, x.z);
        vel[i] = v;
        pos[i] = x;
    }
}

void launch_kick_drift(float4* pos, float4* vel, const float4* acc, int n, float dt_kick, float dt_drift, int grid,
                       cudaStream_t s)
{
    if (n <= 0) return;
    bh_kick_drift_kernel<<<grid, 256, 0, s>>>(pos, vel, acc, n, dt_kick, dt_drift);
}

}  // namespace bh

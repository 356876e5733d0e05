// bh_static.cu -- a force evaluation that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured (allocation is illegal during capture), plugins whose host
// application owns all device memory through its own pool, and real-time
// loops that must not allocate or fail on allocation.  bh_tree_force_static
// serves them: it runs the same kernels as tree_build + tree_moments +
// tree_force, with every work array carved out of one file-scope device
// array of fixed size instead of a context's cudaMalloc'd slab.
//
// The array is a host-side symbol in host code, not a device address, so
// the first call on each device (with that device current) looks up its
// device address with cudaGetSymbolAddress and clears it; that first call
// must come before any stream capture.  All calls share the array and it
// keeps the last call's contents, so calls that overlap on the GPU (two
// streams, two host threads on one device) race and must be serialised by
// the caller.  Every GPU that loads the library holds the array until the
// process exits.
#include <cmath>
#include <cstring>
#include <mutex>

#include "bh_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_bh_static_scratch[BH_STATIC_SCRATCH_BYTES];

struct StaticDevice {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of g_bh_static_scratch on this device
    int sm_count = 1;
};
constexpr int kMaxDevices = 64;
StaticDevice g_static[kMaxDevices];
std::mutex g_static_mu;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool dev_ptr_ok(const void* p, int device)
{
    if (!p || ((uintptr_t)p & 15u)) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace

extern "C" int bh_tree_force_static(const float* d_pos_mass, int64_t n, const bh_config* cfg, float theta,
                                    float eps, float* d_acc_pot, int* h_status, void* stream)
{
    bh_config c;
    if (cfg) {
        c = *cfg;
    } else {
        std::memset(&c, 0, sizeof(c));
        c.leaf_size = 8;
        c.group_size = 64;
        c.order = 1;
        c.fp64_node_threshold = 4096;
        c.block_threads = 128;
        c.max_level = 10;
    }
    if (c.leaf_size < 1 || c.leaf_size > 64 || c.group_size < 1 || c.group_size > 256 ||
        (c.order != 1 && c.order != 2) || c.fp64_node_threshold < 1 ||
        (c.block_threads != 64 && c.block_threads != 128) || c.blocks_per_sm < 0 ||
        c.blocks_per_sm > 32 || (c.curve != BH_CURVE_MORTON && c.curve != BH_CURVE_HILBERT) ||
        c.max_level != 10 ||  // the fixed scratch holds 30-bit keys only
        (c.walk_variant != BH_WALK_ONE_WARP && c.walk_variant != BH_WALK_PAIRED &&
         c.walk_variant != BH_WALK_TMA))  // TMA: no walk records kept here, the one-warp kernel runs
        return BH_ERR_INVALID;
    if (n < 0 || !(theta > 0.0f) || !std::isfinite(theta) || !(eps >= 0.0f) || !std::isfinite(eps))
        return BH_ERR_INVALID;
    if (n > BH_STATIC_MAX_N) return BH_ERR_TOO_LARGE;

    // carve the work arrays for n particles out of the fixed array
    const size_t N = (size_t)(n > 0 ? n : 1);
    const size_t NN = N + 10 * (N / (size_t)(c.leaf_size + 1)) + 1;
    const size_t tiles = (N + bh::kSortTile - 1) / bh::kSortTile;
    const size_t lvl_blocks = (N + bh::kLevelTile - 1) / bh::kLevelTile;
    const size_t flag_blocks = (N + bh::kFlagTile - 1) / bh::kFlagTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_ctrl = take(sizeof(bh_dev_ctrl));
    // look-back words: fixed place and size (the most tiles any call uses), so
    // no other array ever overwrites them; cleared once per device
    const size_t max_tiles = ((size_t)BH_STATIC_MAX_N + bh::kSortTile - 1) / bh::kSortTile;
    const size_t o_look = take(max_tiles * 256 * sizeof(unsigned long long));
    (void)tiles;
    const size_t o_pos = take(N * sizeof(float4));
    const size_t o_keys = take(N * 4), o_keys2 = take(N * 4), o_vals = take(N * 4), o_vals2 = take(N * 4);
    const size_t o_dl = take(N * 2);
    const size_t o_blk = take((lvl_blocks * 11 > flag_blocks ? lvl_blocks * 11 : flag_blocks) * 4);
    const size_t o_flags = take(flag_blocks * bh::kFlagTile);
    const size_t o_gf = take(N * 4), o_gc = take(N * 4);
    const size_t o_first = take(NN * 4), o_count = take(NN * 4), o_child = take(NN * 4), o_nch = take(NN * 4);
    const size_t o_level = take(NN);
    const size_t o_rec = take(NN * sizeof(int4));
    const size_t o_com = take(NN * sizeof(float4));
    const size_t o_seff = take(NN * 4);
    const size_t o_quad = c.order >= 2 ? take(NN * 2 * sizeof(float4)) : 0;
    const size_t o_com64 = take(NN * sizeof(bh_double4));
    const size_t o_quad64 = c.order >= 2 ? take(NN * 6 * sizeof(double)) : 0;
    if (off > (size_t)BH_STATIC_SCRATCH_BYTES) return BH_ERR_TOO_LARGE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return BH_ERR_CUDA;
    }
    if (n > 0 && (!dev_ptr_ok(d_pos_mass, dev) || !dev_ptr_ok(d_acc_pot, dev))) return BH_ERR_INVALID;

    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticDevice& sd = g_static[dev];
    if (!sd.ready) {
        // once per device, with it current: the array's device address, cleared
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bh_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return BH_ERR_CUDA;
        }
        if (cudaMemset(p, 0, BH_STATIC_SCRATCH_BYTES) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            cudaGetLastError();
            return BH_ERR_CUDA;
        }
        cudaDeviceGetAttribute(&sd.sm_count, cudaDevAttrMultiProcessorCount, dev);
        sd.base = (unsigned char*)p;
        sd.ready = true;
    }
    if (n == 0) {
        if (h_status) *h_status = BH_OK;
        return BH_OK;
    }
    unsigned char* b = sd.base;
    bh_dev_ctrl* ctrl = (bh_dev_ctrl*)(b + o_ctrl);
    float4* pos_s = (float4*)(b + o_pos);
    uint32_t* keys = (uint32_t*)(b + o_keys);
    uint32_t* keys_alt = (uint32_t*)(b + o_keys2);
    uint32_t* vals = (uint32_t*)(b + o_vals);
    uint32_t* vals_alt = (uint32_t*)(b + o_vals2);
    int32_t* g_first = (int32_t*)(b + o_gf);
    int32_t* g_count = (int32_t*)(b + o_gc);
    bh_nodes nd;
    nd.first = (int32_t*)(b + o_first);
    nd.count = (int32_t*)(b + o_count);
    nd.child = (int32_t*)(b + o_child);
    nd.nchild = (int32_t*)(b + o_nch);
    nd.level = (uint8_t*)(b + o_level);
    nd.rec = (int4*)(b + o_rec);
    nd.com_m = (float4*)(b + o_com);
    nd.seff = (float*)(b + o_seff);
    nd.quad = c.order >= 2 ? (float4*)(b + o_quad) : nullptr;
    nd.com64 = (bh_double4*)(b + o_com64);
    nd.quad64 = c.order >= 2 ? (double*)(b + o_quad64) : nullptr;

    cudaStream_t s = (cudaStream_t)stream;
    const int N32 = (int)n;
    const int grid = sd.sm_count * 8;
    const float4* pos = (const float4*)d_pos_mass;
    bh::launch_init(ctrl, s);
    bh::launch_bbox(pos, N32, ctrl, grid, s);
    bh::launch_keys(pos, N32, ctrl, keys, c.curve, false, grid, s);
    bh::launch_sort(keys, keys_alt, vals, vals_alt, pos, pos_s, N32, (unsigned long long*)(b + o_look), ctrl,
                    false, s);
    bh::launch_tree(keys, false, N32, c.leaf_size, (uint16_t*)(b + o_dl), (uint32_t*)(b + o_blk), nd, (int64_t)NN,
                    ctrl, grid, s);
    bh::launch_groups(nd, N32, c.group_size, (uint8_t*)(b + o_flags), (uint32_t*)(b + o_blk), g_first, g_count,
                      ctrl, grid, s);
    bh::launch_moments(pos_s, keys, false, nd, c.order, theta, c.fp64_node_threshold, c.curve, ctrl, grid, s);
    int rc = bh::launch_walk(pos_s, vals, g_first, g_count, nd, c.order, c.group_size, eps, (float4*)d_acc_pot, ctrl,
                             sd.sm_count, c.block_threads, c.blocks_per_sm, s, nullptr, c.walk_variant);
    if (rc) return rc;
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    if (h_status) {
        unsigned int st = 0u;
        if (cudaMemcpyAsync(&st, &ctrl->status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return BH_ERR_CUDA;
        *h_status = -(int)st;
    }
    return BH_OK;
}

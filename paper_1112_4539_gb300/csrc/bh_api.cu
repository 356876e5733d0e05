// bh_api.cu -- the C ABI of libbhtree (declared in include/bhtree.h).
//
// A context owns one device slab holding every work array for up to max_n
// particles, so tree_build / tree_moments / tree_force allocate nothing and
// never synchronise: the whole evaluation is stream-ordered and can be
// captured in a CUDA graph.  Device-side failures land in the control block's
// status word, read back by bh_status / bh_stats.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "bh_mlp.cuh"

struct bh_ctx {
    int device = 0;
    int sm_count = 1;
    bh_config cfg{};
    int64_t max_n = 0;
    int64_t node_cap = 0;
    bool deep = false;  // 63-bit keys (21 levels) instead of 30-bit keys (10 levels)
    int64_t n = -1;  // particles of the last tree_build (-1: none)
    bool have_moments = false;
    float theta = 0.f;
    int64_t launches = 0;
    void* slab = nullptr;
    bh_dev_ctrl* ctrl = nullptr;
    bh_dev_ctrl* host_ctrl = nullptr;  // pinned staging for read-back
    float4* pos_s = nullptr;
    void *keys = nullptr, *keys_alt = nullptr;   // uint32_t[n] or, deep, uint64_t[n]
    uint32_t *vals = nullptr, *vals_alt = nullptr;
    unsigned long long* lookback = nullptr;
    uint16_t* dl = nullptr;
    uint32_t* blk = nullptr;
    uint8_t* flags = nullptr;
    int32_t *g_first = nullptr, *g_count = nullptr;
    bh_nodes nd{};
    // learned opening criterion
    bool mac_learned = false;
    float4* mfeat = nullptr;        // node-constant features
    bh_mlp_dev* mlp = nullptr;      // packed network (device)
    // several independent systems
    int nsys = 0;                   // systems of the current layout (0: none)
    int64_t batch_n = 0;            // their total particle count
    uint32_t* sys_of = nullptr;     // system of each Morton position
    int32_t* sys_off = nullptr;     // first particle of each system (+ total)
    float4* sys_box = nullptr;      // root cube of each system
    // links of the per-particle walk
    int32_t* parent = nullptr;
    int32_t* next = nullptr;
    // node bounding boxes of the neighbour search
    float4* blo = nullptr;
    float4* bhi = nullptr;
    // individual softening (allocated by the first tree_softening call)
    void* soft_slab = nullptr;
    bh::bh_soft soft{};
    bool have_soft = false;
};

namespace {

int grid_for(const bh_ctx* c) { return c->sm_count * 8; }

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// true if p is a device pointer usable on `device` (device or managed memory)
bool is_device_ptr(const void* p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int d)
    {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" {

int bh_version(void) { return 10000; }

const char* bh_strerror(int code)
{
    switch (code) {
        case BH_OK: return "ok";
        case BH_ERR_INVALID: return "invalid argument";
        case BH_ERR_TOO_LARGE: return "size exceeds a limit";
        case BH_ERR_NONFINITE: return "non-finite particle coordinate or mass";
        case BH_ERR_CAPACITY: return "device work list capacity exceeded";
        case BH_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
        case BH_ERR_CUDA: return "CUDA runtime error";
        case BH_ERR_STATE: return "call order violated";
        case BH_ERR_NOMEM: return "device allocation failed";
        default: return "unknown error";
    }
}

void bh_config_default(bh_config* cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->leaf_size = 8;
    cfg->group_size = 64;
    cfg->order = 1;
    cfg->fp64_node_threshold = 4096;
    cfg->block_threads = 128;
    cfg->blocks_per_sm = 0;
    cfg->max_systems = 1;
    cfg->curve = BH_CURVE_MORTON;
    cfg->max_level = 10;
    cfg->walk_variant = BH_WALK_ONE_WARP;
}

static int validate_config(const bh_config* c)
{
    if (c->leaf_size < 1 || c->leaf_size > 64) return BH_ERR_INVALID;
    if (c->group_size < 1 || c->group_size > 256) return BH_ERR_INVALID;
    if (c->order != 1 && c->order != 2) return BH_ERR_INVALID;
    if (c->fp64_node_threshold < 1) return BH_ERR_INVALID;
    if (c->block_threads != 64 && c->block_threads != 128) return BH_ERR_INVALID;
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > 32) return BH_ERR_INVALID;
    if (c->max_systems < 0 || c->max_systems > (1 << 20)) return BH_ERR_INVALID;
    if (c->curve != BH_CURVE_MORTON && c->curve != BH_CURVE_HILBERT) return BH_ERR_INVALID;
    if (c->max_level != 10 && c->max_level != 21) return BH_ERR_INVALID;
    if (c->walk_variant != BH_WALK_ONE_WARP && c->walk_variant != BH_WALK_PAIRED && c->walk_variant != BH_WALK_TMA)
        return BH_ERR_INVALID;
    return BH_OK;
}

int bh_create(bh_ctx** out, const bh_config* cfg, int64_t max_n, int device)
{
    if (!out) return BH_ERR_INVALID;
    *out = nullptr;
    bh_config c;
    if (cfg) c = *cfg;
    else bh_config_default(&c);
    int rc = validate_config(&c);
    if (rc) return rc;
    if (max_n < 1) return BH_ERR_INVALID;
    if (max_n >= (int64_t)1 << 30) return BH_ERR_TOO_LARGE;
    // <= max_n leaves plus, on each level above the deepest, <= max_n / (leaf_size + 1) internal nodes
    const int64_t node_cap = max_n + (int64_t)c.max_level * (max_n / (c.leaf_size + 1)) + 1;
    if (node_cap >= (int64_t)1 << 28) return BH_ERR_TOO_LARGE;  // walk stack packs node ids in 28 bits
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return BH_ERR_INVALID;
    }
    DeviceGuard guard(device);
    bh_ctx* x = new (std::nothrow) bh_ctx();
    if (!x) return BH_ERR_NOMEM;
    x->device = device;
    x->cfg = c;
    x->max_n = max_n;
    x->node_cap = node_cap;
    x->deep = c.max_level == BH_MAX_LEVEL_DEEP;
    cudaDeviceGetAttribute(&x->sm_count, cudaDevAttrMultiProcessorCount, device);

    const size_t N = (size_t)max_n, NN = (size_t)node_cap;
    const int tile = x->deep ? bh::kSortTileDeep : bh::kSortTile;
    const size_t sort_tiles = (N + tile - 1) / tile;
    const size_t kb = x->deep ? 8 : 4, nlev = (size_t)c.max_level + 1;
    const size_t lvl_blocks = (N + bh::kLevelTile - 1) / bh::kLevelTile;
    const size_t flag_blocks = (N + bh::kFlagTile - 1) / bh::kFlagTile;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t o_ctrl = take(sizeof(bh_dev_ctrl));
    const size_t o_pos = take(N * sizeof(float4));
    const size_t o_keys = take(N * kb), o_keys2 = take(N * kb), o_vals = take(N * 4), o_vals2 = take(N * 4);
    const size_t o_look = take(sort_tiles * 256 * sizeof(unsigned long long));
    const size_t o_dl = take(N * 2);
    const size_t o_blk = take(std::max(lvl_blocks * nlev, flag_blocks) * 4);
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
    // walk records exist only for the TMA-staged walk (the moments pass writes them when present)
    const size_t o_wrec = c.walk_variant == BH_WALK_TMA ? take(NN * bh_wrec_f4(c.order) * sizeof(float4)) : 0;
    const size_t o_mfeat = take(NN * sizeof(float4));
    const size_t o_mlp = take(sizeof(bh_mlp_dev));
    const size_t S = (size_t)std::max(1, c.max_systems);
    const size_t o_sys = take(N * 4), o_soff = take((S + 1) * 4), o_sbox = take(S * sizeof(float4));
    const size_t o_parent = take(NN * 4), o_next = take(NN * 4);
    const size_t o_blo = take(NN * sizeof(float4)), o_bhi = take(NN * sizeof(float4));
    const size_t total = off;

    if (cudaMalloc(&x->slab, total) != cudaSuccess) {
        cudaGetLastError();
        delete x;
        return BH_ERR_NOMEM;
    }
    if (cudaMallocHost((void**)&x->host_ctrl, sizeof(bh_dev_ctrl)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(x->slab);
        delete x;
        return BH_ERR_NOMEM;
    }
    char* b = (char*)x->slab;
    x->ctrl = (bh_dev_ctrl*)(b + o_ctrl);
    x->pos_s = (float4*)(b + o_pos);
    x->keys = (void*)(b + o_keys);
    x->keys_alt = (void*)(b + o_keys2);
    x->vals = (uint32_t*)(b + o_vals);
    x->vals_alt = (uint32_t*)(b + o_vals2);
    x->lookback = (unsigned long long*)(b + o_look);
    x->dl = (uint16_t*)(b + o_dl);
    x->blk = (uint32_t*)(b + o_blk);
    x->flags = (uint8_t*)(b + o_flags);
    x->g_first = (int32_t*)(b + o_gf);
    x->g_count = (int32_t*)(b + o_gc);
    x->nd.first = (int32_t*)(b + o_first);
    x->nd.count = (int32_t*)(b + o_count);
    x->nd.child = (int32_t*)(b + o_child);
    x->nd.nchild = (int32_t*)(b + o_nch);
    x->nd.level = (uint8_t*)(b + o_level);
    x->nd.rec = (int4*)(b + o_rec);
    x->nd.com_m = (float4*)(b + o_com);
    x->nd.seff = (float*)(b + o_seff);
    x->nd.quad = c.order >= 2 ? (float4*)(b + o_quad) : nullptr;
    x->nd.com64 = (bh_double4*)(b + o_com64);
    x->nd.quad64 = c.order >= 2 ? (double*)(b + o_quad64) : nullptr;
    x->nd.wrec = c.walk_variant == BH_WALK_TMA ? (float4*)(b + o_wrec) : nullptr;
    x->mfeat = (float4*)(b + o_mfeat);
    x->mlp = (bh_mlp_dev*)(b + o_mlp);
    x->sys_of = (uint32_t*)(b + o_sys);
    x->sys_off = (int32_t*)(b + o_soff);
    x->sys_box = (float4*)(b + o_sbox);
    x->parent = (int32_t*)(b + o_parent);
    x->next = (int32_t*)(b + o_next);
    x->blo = (float4*)(b + o_blo);
    x->bhi = (float4*)(b + o_bhi);
    if (x->cfg.max_systems < 1) x->cfg.max_systems = 1;
    // look-back words start at epoch 0, which no pass uses; control block zeroed
    if (cudaMemset(x->lookback, 0, sort_tiles * 256 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(x->ctrl, 0, sizeof(bh_dev_ctrl)) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(x->host_ctrl);
        cudaFree(x->slab);
        delete x;
        return BH_ERR_CUDA;
    }
    *out = x;
    return BH_OK;
}

void bh_destroy(bh_ctx* x)
{
    if (!x) return;
    DeviceGuard guard(x->device);
    cudaDeviceSynchronize();
    cudaFreeHost(x->host_ctrl);
    cudaFree(x->slab);
    if (x->soft_slab) cudaFree(x->soft_slab);
    delete x;
}

int tree_build(bh_ctx* x, const float* d_pos_mass, int64_t n, void* stream)
{
    if (!x) return BH_ERR_INVALID;
    if (n < 0) return BH_ERR_INVALID;
    if (n > x->max_n) return BH_ERR_TOO_LARGE;
    if (n > 0 && (!d_pos_mass || !aligned16(d_pos_mass) || !is_device_ptr(d_pos_mass, x->device)))
        return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int N = (int)n;
    const float4* pos = (const float4*)d_pos_mass;
    bh::launch_init(x->ctrl, s);
    if (N > 0) {
        bh::launch_bbox(pos, N, x->ctrl, grid_for(x), s);
        bh::launch_keys(pos, N, x->ctrl, x->keys, x->cfg.curve, x->deep, grid_for(x), s);
        bh::launch_sort(x->keys, x->keys_alt, x->vals, x->vals_alt, pos, x->pos_s, N, x->lookback, x->ctrl,
                        x->deep, s);
        bh::launch_tree(x->keys, x->deep, N, x->cfg.leaf_size, x->dl, x->blk, x->nd, x->node_cap, x->ctrl,
                        grid_for(x), s);
        bh::launch_groups(x->nd, N, x->cfg.group_size, x->flags, x->blk, x->g_first, x->g_count, x->ctrl,
                          grid_for(x), s);
        x->launches += bh::launches_build(x->deep) - 1;
    }
    x->launches += 1;
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    x->n = n;
    x->have_moments = false;
    x->have_soft = false;
    return BH_OK;
}

int tree_softening(bh_ctx* x, const float* d_eps, void* stream)
{
    if (!x) return BH_ERR_INVALID;
    if (x->n < 0) return BH_ERR_STATE;
    if (x->n > 0 && (!d_eps || ((uintptr_t)d_eps & 3u) || !is_device_ptr(d_eps, x->device))) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    if (!x->soft_slab) {
        const size_t a = ((size_t)x->max_n * sizeof(float) + 255) & ~(size_t)255;
        const size_t b = ((size_t)x->node_cap * sizeof(double2) + 255) & ~(size_t)255;
        if (cudaMalloc(&x->soft_slab, a + b + (size_t)x->node_cap * sizeof(float) + 256) != cudaSuccess) {
            cudaGetLastError();
            x->soft_slab = nullptr;
            return BH_ERR_NOMEM;
        }
        unsigned char* p = (unsigned char*)x->soft_slab;
        x->soft.h = (float*)p;
        x->soft.sums = (double2*)(p + a);
        x->soft.hbar = (float*)(p + a + b);
    }
    if (x->n > 0) {
        bh::launch_softening(d_eps, x->vals, x->pos_s, x->nd, (int)x->n, x->deep, x->soft, x->ctrl, grid_for(x),
                             (cudaStream_t)stream);
        x->launches += bh::launches_softening(x->deep);
    }
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    x->have_soft = true;
    return BH_OK;
}

int tree_moments(bh_ctx* x, float theta, void* stream)
{
    if (!x) return BH_ERR_INVALID;
    if (!(theta > 0.0f) || !std::isfinite(theta)) return BH_ERR_INVALID;
    if (x->n < 0) return BH_ERR_STATE;
    DeviceGuard guard(x->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (x->n > 0) {
        bh::launch_moments(x->pos_s, x->keys, x->deep, x->nd, x->cfg.order, theta, x->cfg.fp64_node_threshold,
                           x->cfg.curve, x->ctrl, grid_for(x), s);
        x->launches += bh::launches_moments(x->deep);
        if (x->mac_learned) {
            bh::launch_mac_nodefeat(x->nd, x->cfg.order, x->mfeat, x->ctrl, grid_for(x), s);
            x->launches += 1;
        }
    }
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    x->theta = theta;
    x->have_moments = true;
    return BH_OK;
}

int tree_force(bh_ctx* x, float eps, float* d_acc_pot, void* stream)
{
    if (!x) return BH_ERR_INVALID;
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return BH_ERR_INVALID;
    if (x->n < 0 || !x->have_moments) return BH_ERR_STATE;
    if (x->n == 0) return BH_OK;
    if (!d_acc_pot || !aligned16(d_acc_pot) || !is_device_ptr(d_acc_pot, x->device)) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    cudaStream_t s = (cudaStream_t)stream;
    bh::WalkLearned wl{x->mfeat, x->mlp, x->theta};
    int rc = bh::launch_walk(x->pos_s, x->vals, x->g_first, x->g_count, x->nd, x->cfg.order, x->cfg.group_size,
                             eps, (float4*)d_acc_pot, x->ctrl, x->sm_count, x->cfg.block_threads,
                             x->cfg.blocks_per_sm, s, x->mac_learned ? &wl : nullptr, x->cfg.walk_variant);
    if (rc) return rc;
    x->launches += bh::kLaunchesForce;
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    return BH_OK;
}

int tree_force_particles(bh_ctx* x, float eps, int flags, float* d_acc_pot, void* stream)
{
    if (!x) return BH_ERR_INVALID;
    if (!(eps >= 0.0f) || !std::isfinite(eps)) return BH_ERR_INVALID;
    if (flags & ~(BH_PWALK_UNSOFTENED_CELLS | BH_PWALK_INDIVIDUAL_SOFTENING)) return BH_ERR_INVALID;
    if (x->n < 0 || !x->have_moments) return BH_ERR_STATE;
    const bool ind = (flags & BH_PWALK_INDIVIDUAL_SOFTENING) != 0;
    if (ind && !x->have_soft) return BH_ERR_STATE;
    if (x->n == 0) return BH_OK;
    if (!d_acc_pot || !aligned16(d_acc_pot) || !is_device_ptr(d_acc_pot, x->device)) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    int rc = bh::launch_pwalk(x->pos_s, x->vals, x->nd, x->parent, x->next, x->cfg.order, (int)x->n,
                              (int)x->node_cap, eps, (flags & BH_PWALK_UNSOFTENED_CELLS) != 0, (float4*)d_acc_pot,
                              x->ctrl, x->sm_count, (cudaStream_t)stream, ind ? &x->soft : nullptr);
    if (rc) return rc;
    x->launches += bh::kLaunchesPWalk;
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    return BH_OK;
}

int tree_neighbors(bh_ctx* x, const float* d_h, float h, int32_t* d_count, float* d_rho, void* stream)
{
    if (!x) return BH_ERR_INVALID;
    if (!d_h && !(h > 0.0f && std::isfinite(h))) return BH_ERR_INVALID;
    if (x->n < 0) return BH_ERR_STATE;
    if (x->n == 0) return BH_OK;
    if (d_h && (((uintptr_t)d_h & 3u) || !is_device_ptr(d_h, x->device))) return BH_ERR_INVALID;
    if (d_count && (((uintptr_t)d_count & 3u) || !is_device_ptr(d_count, x->device))) return BH_ERR_INVALID;
    if (d_rho && (((uintptr_t)d_rho & 3u) || !is_device_ptr(d_rho, x->device))) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    int rc = bh::launch_sph(x->pos_s, x->vals, x->g_first, x->g_count, x->nd, x->blo, x->bhi, x->cfg.group_size, d_h,
                            h, d_count, d_rho, x->ctrl, x->sm_count, grid_for(x), x->cfg.max_level,
                            (cudaStream_t)stream);
    if (rc) return rc;
    x->launches += bh::launches_sph(x->deep);
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    return BH_OK;
}

int bh_kick_drift(bh_ctx* x, float* d_pos, float* d_vel, const float* d_acc, int64_t n, float dt_kick,
                  float dt_drift, void* stream)
{
    if (!x || n < 0) return BH_ERR_INVALID;
    if (n >= ((int64_t)1 << 31)) return BH_ERR_TOO_LARGE;
    if (n == 0) return BH_OK;
    for (const void* p : {(const void*)d_pos, (const void*)d_vel, (const void*)d_acc})
        if (!p || !aligned16(p) || !is_device_ptr(p, x->device)) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    bh::launch_kick_drift((float4*)d_pos, (float4*)d_vel, (const float4*)d_acc, (int)n, dt_kick, dt_drift,
                          grid_for(x), (cudaStream_t)stream);
    x->launches += 1;
    return cudaGetLastError() == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

int direct_force(const float* d_src, int64_t n_src, const float* d_tgt, const int64_t* d_tgt_self, int64_t n_tgt,
                 double eps, void* d_out, int precision, void* stream)
{
    if (n_src < 0 || n_tgt < 0) return BH_ERR_INVALID;
    if (n_src >= ((int64_t)1 << 31) || n_tgt >= ((int64_t)1 << 31)) return BH_ERR_TOO_LARGE;
    if (precision != 32 && precision != 64) return BH_ERR_INVALID;
    if (!(eps >= 0.0) || !std::isfinite(eps)) return BH_ERR_INVALID;
    if (n_tgt == 0) return BH_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BH_ERR_CUDA;
    if (!d_tgt || !aligned16(d_tgt) || !is_device_ptr(d_tgt, dev)) return BH_ERR_INVALID;
    if (!d_out || !aligned16(d_out) || !is_device_ptr(d_out, dev)) return BH_ERR_INVALID;
    if (n_src > 0 && (!d_src || !aligned16(d_src) || !is_device_ptr(d_src, dev))) return BH_ERR_INVALID;
    if (d_tgt_self && (((uintptr_t)d_tgt_self & 7u) || !is_device_ptr(d_tgt_self, dev))) return BH_ERR_INVALID;
    return bh::launch_direct((const float4*)d_src, (int)n_src, (const float4*)d_tgt, d_tgt_self, (int)n_tgt, eps,
                             d_out, precision, (cudaStream_t)stream);
}

int direct_force_sym(const float* d_src, const float* d_eps_src, int64_t n_src, const float* d_tgt,
                     const float* d_eps_tgt, const int64_t* d_tgt_self, int64_t n_tgt, void* d_out, int precision,
                     void* stream)
{
    if (n_src < 0 || n_tgt < 0) return BH_ERR_INVALID;
    if (n_src >= ((int64_t)1 << 31) || n_tgt >= ((int64_t)1 << 31)) return BH_ERR_TOO_LARGE;
    if (precision != 32 && precision != 64) return BH_ERR_INVALID;
    if (n_tgt == 0) return BH_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BH_ERR_CUDA;
    if (!d_tgt || !aligned16(d_tgt) || !is_device_ptr(d_tgt, dev)) return BH_ERR_INVALID;
    if (!d_out || !aligned16(d_out) || !is_device_ptr(d_out, dev)) return BH_ERR_INVALID;
    if (!d_eps_tgt || ((uintptr_t)d_eps_tgt & 3u) || !is_device_ptr(d_eps_tgt, dev)) return BH_ERR_INVALID;
    if (n_src > 0 && (!d_src || !aligned16(d_src) || !is_device_ptr(d_src, dev))) return BH_ERR_INVALID;
    if (n_src > 0 && (!d_eps_src || ((uintptr_t)d_eps_src & 3u) || !is_device_ptr(d_eps_src, dev)))
        return BH_ERR_INVALID;
    if (d_tgt_self && (((uintptr_t)d_tgt_self & 7u) || !is_device_ptr(d_tgt_self, dev))) return BH_ERR_INVALID;
    // (n_src == 0 only zeroes the output)
    return bh::launch_direct((const float4*)d_src, (int)n_src, (const float4*)d_tgt, d_tgt_self, (int)n_tgt, 0.0,
                             d_out, precision, (cudaStream_t)stream, d_eps_src, d_eps_tgt);
}

static int read_ctrl(bh_ctx* x, cudaStream_t s)
{
    if (cudaMemcpyAsync(x->host_ctrl, x->ctrl, sizeof(bh_dev_ctrl), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return BH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BH_ERR_CUDA;
    return BH_OK;
}

int bh_selftest_wait(bh_ctx* x, int which, void* stream)
{
    if (!x || (which != BH_SELFTEST_TILE_RING && which != BH_SELFTEST_LOOKBACK && which != BH_SELFTEST_TMA))
        return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (which == BH_SELFTEST_TILE_RING) bh::launch_selftest_ring(x->ctrl, s);
    else if (which == BH_SELFTEST_TMA) bh::launch_selftest_tma(x->ctrl, s);
    else bh::launch_selftest_lookback(x->ctrl, s);
    x->launches += 1;
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    return BH_OK;
}

int bh_status(bh_ctx* x, void* stream)
{
    if (!x) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = read_ctrl(x, s);
    if (rc) return rc;
    const int st = -(int)x->host_ctrl->status;
    if (st != 0) {
        const unsigned int zero[2] = {0u, 0u};
        cudaMemcpyAsync(&x->ctrl->status, zero, sizeof(zero), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
    }
    return st;
}

int bh_stats(bh_ctx* x, void* stream, bh_stats_t* out)
{
    if (!x || !out) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    int rc = read_ctrl(x, (cudaStream_t)stream);
    if (rc) return rc;
    const bh_dev_ctrl& h = *x->host_ctrl;
    std::memset(out, 0, sizeof(*out));
    out->n = x->n < 0 ? 0 : x->n;
    out->n_nodes = h.n_nodes;
    out->n_leaves = h.n_leaves;
    out->n_groups = h.n_groups;
    out->n_pp = (int64_t)h.n_pp;
    out->n_pc = (int64_t)h.n_pc;
    out->max_leaf_count = h.max_leaf;
    out->status = -(int)h.status;
    for (int i = 0; i < 4; i++) out->box[i] = h.box[i];
    out->n_pp_total = (int64_t)h.cum_pp;
    out->n_pc_total = (int64_t)h.cum_pc;
    out->launches = x->launches;
    return BH_OK;
}

int bh_export(bh_ctx* x, int what, void* dst, int64_t cap_bytes, int64_t* out_bytes, void* stream)
{
    if (!x || !dst) return BH_ERR_INVALID;
    if (x->n < 0) return BH_ERR_STATE;
    DeviceGuard guard(x->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = read_ctrl(x, s);
    if (rc) return rc;
    const int64_t n = x->n, nn = x->host_ctrl->n_nodes, ng = x->host_ctrl->n_groups;
    const void* src = nullptr;
    int64_t bytes = 0;
    switch (what) {
        case BH_EXPORT_KEYS: src = x->keys; bytes = n * (x->deep ? 8 : 4); break;
        case BH_EXPORT_PERM: src = x->vals; bytes = n * 4; break;
        case BH_EXPORT_SPOS: src = x->pos_s; bytes = n * 16; break;
        case BH_EXPORT_NODE_FIRST: src = x->nd.first; bytes = nn * 4; break;
        case BH_EXPORT_NODE_COUNT: src = x->nd.count; bytes = nn * 4; break;
        case BH_EXPORT_NODE_CHILD: src = x->nd.child; bytes = nn * 4; break;
        case BH_EXPORT_NODE_NCHILD: src = x->nd.nchild; bytes = nn * 4; break;
        case BH_EXPORT_NODE_LEVEL: src = nullptr; bytes = nn * 4; break;
        case BH_EXPORT_COM_M: src = x->nd.com_m; bytes = nn * 16; break;
        case BH_EXPORT_SEFF: src = x->nd.seff; bytes = nn * 4; break;
        case BH_EXPORT_QUAD:
            if (x->cfg.order < 2) return BH_ERR_STATE;
            src = nullptr;
            bytes = nn * 24;
            break;
        case BH_EXPORT_GROUP_FIRST: src = x->g_first; bytes = ng * 4; break;
        case BH_EXPORT_GROUP_COUNT: src = x->g_count; bytes = ng * 4; break;
        case BH_EXPORT_BOX: src = x->ctrl->box; bytes = 16; break;
        case BH_EXPORT_NEXT: src = x->next; bytes = nn * 4; break;
        default: return BH_ERR_INVALID;
    }
    if (out_bytes) *out_bytes = bytes;
    if (cap_bytes < bytes) return BH_ERR_TOO_LARGE;
    if (bytes == 0) return BH_OK;
    if (what == BH_EXPORT_NODE_LEVEL || what == BH_EXPORT_QUAD) {
        // widen / unpack through a host copy
        const bool lev = what == BH_EXPORT_NODE_LEVEL;
        const size_t hb = lev ? (size_t)nn : (size_t)nn * 32;
        void* h = std::malloc(hb ? hb : 1);
        if (!h) return BH_ERR_NOMEM;
        void* hout = std::malloc((size_t)bytes);
        if (!hout) {
            std::free(h);
            return BH_ERR_NOMEM;
        }
        cudaMemcpyAsync(h, lev ? (const void*)x->nd.level : (const void*)x->nd.quad, hb, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            std::free(h);
            std::free(hout);
            return BH_ERR_CUDA;
        }
        if (lev) {
            for (int64_t i = 0; i < nn; i++) ((int32_t*)hout)[i] = ((const uint8_t*)h)[i];
        } else {
            const float* q = (const float*)h;
            float* o = (float*)hout;
            for (int64_t i = 0; i < nn; i++)
                for (int k = 0; k < 6; k++) o[6 * i + k] = q[8 * i + k];
        }
        const cudaError_t e = cudaMemcpy(dst, hout, (size_t)bytes, cudaMemcpyDefault);
        std::free(h);
        std::free(hout);
        return e == cudaSuccess ? BH_OK : BH_ERR_CUDA;
    }
    if (cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDefault, s) != cudaSuccess) return BH_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return BH_ERR_CUDA;
    return BH_OK;
}

// ------------------------------------------------------------------ learned criterion
int bh_mac_set(bh_ctx* x, const float* h_params, const float* h_fmin, const float* h_fmax, float tau,
               float theta_fb)
{
    if (!x) return BH_ERR_INVALID;
    if (!h_params) {
        x->mac_learned = false;
        x->have_moments = false;
        return BH_OK;
    }
    if (!h_fmin || !h_fmax || !(tau > 0.0f) || !std::isfinite(tau) || !(theta_fb > 0.0f) || !std::isfinite(theta_fb))
        return BH_ERR_INVALID;
    for (int k = 0; k < BH_MLP_NPARAM; k++)
        if (!std::isfinite(h_params[k])) return BH_ERR_INVALID;
    bh_mlp_dev host;
    bh::mlp_pack(h_params, h_fmin, h_fmax, std::log10(tau), theta_fb, &host);
    DeviceGuard guard(x->device);
    // the packed copy may be read by enqueued walks: wait for them first
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(x->mlp, &host, sizeof(host), cudaMemcpyHostToDevice) !=
                                                      cudaSuccess)
        return BH_ERR_CUDA;
    x->mac_learned = true;
    x->have_moments = false;  // node features are computed by the next tree_moments
    return BH_OK;
}

int bh_mac_label(bh_ctx* x, const int32_t* d_groups, int64_t n_groups, const float* d_acc_ref, float eps,
                 float log10_floor, float* d_X, float* d_Y, int32_t* d_pairs, int64_t cap,
                 unsigned long long* d_count, void* stream)
{
    if (d_pairs && x && !is_device_ptr(d_pairs, x->device)) return BH_ERR_INVALID;
    if (!x || n_groups < 0 || cap < 0 || !(eps >= 0.0f) || !std::isfinite(eps)) return BH_ERR_INVALID;
    if (x->n < 0 || !x->have_moments) return BH_ERR_STATE;
    if (n_groups >= ((int64_t)1 << 31)) return BH_ERR_TOO_LARGE;
    if (n_groups == 0 || x->n == 0) return BH_OK;
    for (const void* p : {(const void*)d_groups, (const void*)d_X, (const void*)d_Y, (const void*)d_count})
        if (!p || !is_device_ptr(p, x->device)) return BH_ERR_INVALID;
    if (!d_acc_ref || !aligned16(d_acc_ref) || !is_device_ptr(d_acc_ref, x->device)) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    cudaStream_t s = (cudaStream_t)stream;
    bh::launch_mac_nodefeat(x->nd, x->cfg.order, x->mfeat, x->ctrl, grid_for(x), s);
    x->launches += 2;
    return bh::mac_label(x->pos_s, x->vals, x->g_first, x->g_count, d_groups, (int)n_groups, x->nd, x->mfeat,
                         (const float4*)d_acc_ref, eps, log10_floor, x->cfg.order, d_X, d_Y, d_pairs, (long long)cap,
                         d_count, x->ctrl, s);
}

int bh_mlp_train(const float* d_X, const float* d_Y, const int32_t* d_order, int64_t n, float* d_params,
                 float* d_adam_m, float* d_adam_v, float* d_work, int64_t work_floats, int64_t steps, int batch,
                 float lr, float under_weight, float* d_loss, int64_t t0, void* stream)
{
    if (n < 1 || steps < 0 || batch < 1 || t0 < 0 || !(lr > 0.0f) || !(under_weight > 0.0f)) return BH_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BH_ERR_CUDA;
    for (const void* p : {(const void*)d_X, (const void*)d_Y, (const void*)d_params, (const void*)d_adam_m,
                          (const void*)d_adam_v, (const void*)d_work})
        if (!p || !is_device_ptr(p, dev)) return BH_ERR_INVALID;
    if (d_order && !is_device_ptr(d_order, dev)) return BH_ERR_INVALID;
    if (d_loss && !is_device_ptr(d_loss, dev)) return BH_ERR_INVALID;
    return bh::mlp_train(d_X, d_Y, d_order, (long long)n, d_params, d_adam_m, d_adam_v, d_work, (long long)work_floats,
                         (long long)steps, batch, lr, under_weight, d_loss, (long long)t0, (cudaStream_t)stream);
}

int bh_mlp_grad(const float* d_params, const float* d_X, const float* d_Y, int64_t n, float under_weight,
                float* d_work, int64_t work_floats, float* d_grad, float* d_loss, void* stream)
{
    if (n < 1 || !(under_weight > 0.0f)) return BH_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BH_ERR_CUDA;
    for (const void* p : {(const void*)d_params, (const void*)d_X, (const void*)d_Y, (const void*)d_work,
                          (const void*)d_grad})
        if (!p || !is_device_ptr(p, dev)) return BH_ERR_INVALID;
    if (d_loss && !is_device_ptr(d_loss, dev)) return BH_ERR_INVALID;
    return bh::mlp_grad(d_params, d_X, d_Y, (long long)n, under_weight, d_work, (long long)work_floats, d_grad,
                        d_loss, (cudaStream_t)stream);
}

int bh_mlp_forward(bh_ctx* x, const float* d_params, const float* d_X, int64_t n, float* d_y, int precision,
                   void* stream)
{
    if (n < 0 || (precision != 16 && precision != 32)) return BH_ERR_INVALID;
    if (n == 0) return BH_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BH_ERR_CUDA;
    if (!d_X || !d_y || !is_device_ptr(d_X, dev) || !is_device_ptr(d_y, dev)) return BH_ERR_INVALID;
    if (precision == 16) {
        if (!x || !x->mac_learned) return BH_ERR_STATE;
        return bh::mlp_forward(nullptr, x->mlp, d_X, (long long)n, d_y, 16, (cudaStream_t)stream);
    }
    if (!d_params || !is_device_ptr(d_params, dev)) return BH_ERR_INVALID;
    return bh::mlp_forward(d_params, nullptr, d_X, (long long)n, d_y, 32, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ many systems
int bh_batch_layout(bh_ctx* x, const int64_t* h_offsets, int nsys)
{
    if (!x || !h_offsets || nsys < 1) return BH_ERR_INVALID;
    if (nsys > x->cfg.max_systems) return BH_ERR_TOO_LARGE;
    if (h_offsets[0] != 0) return BH_ERR_INVALID;
    std::vector<int32_t> off32((size_t)nsys + 1);
    for (int s = 0; s < nsys; s++) {
        const int64_t c = h_offsets[s + 1] - h_offsets[s];
        if (c < 0) return BH_ERR_INVALID;
        if (c > bh::kBatchMaxN) return BH_ERR_TOO_LARGE;
        off32[(size_t)s] = (int32_t)h_offsets[s];
    }
    if (h_offsets[nsys] > x->max_n) return BH_ERR_TOO_LARGE;
    off32[(size_t)nsys] = (int32_t)h_offsets[nsys];
    DeviceGuard guard(x->device);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(x->sys_off, off32.data(), off32.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        return BH_ERR_CUDA;
    x->nsys = nsys;
    x->batch_n = h_offsets[nsys];
    return BH_OK;
}

int bh_force_batched(bh_ctx* x, const float* d_pos_mass, float theta, float eps, float* d_acc_pot, void* stream)
{
    if (!x) return BH_ERR_INVALID;
    if (x->nsys < 1 || x->mac_learned) return BH_ERR_STATE;
    if (!(theta > 0.0f) || !std::isfinite(theta) || !(eps >= 0.0f) || !std::isfinite(eps)) return BH_ERR_INVALID;
    const int64_t n = x->batch_n;
    if (n == 0) return BH_OK;
    if (!d_pos_mass || !aligned16(d_pos_mass) || !is_device_ptr(d_pos_mass, x->device)) return BH_ERR_INVALID;
    if (!d_acc_pot || !aligned16(d_acc_pot) || !is_device_ptr(d_acc_pot, x->device)) return BH_ERR_INVALID;
    DeviceGuard guard(x->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int N = (int)n;
    bh::launch_init(x->ctrl, s);
    bh::launch_batch_sort((const float4*)d_pos_mass, x->sys_off, x->nsys, x->keys, x->keys_alt, x->vals, x->vals_alt,
                          x->pos_s, x->sys_of, x->sys_box, x->cfg.curve, x->deep, x->ctrl, s);
    bh::launch_tree(x->keys, x->deep, N, x->cfg.leaf_size, x->dl, x->blk, x->nd, x->node_cap, x->ctrl, grid_for(x),
                    s, x->sys_of, x->sys_off);
    bh::launch_groups(x->nd, N, x->cfg.group_size, x->flags, x->blk, x->g_first, x->g_count, x->ctrl, grid_for(x), s);
    bh::launch_moments(x->pos_s, x->keys, x->deep, x->nd, x->cfg.order, theta, x->cfg.fp64_node_threshold,
                       x->cfg.curve, x->ctrl, grid_for(x), s, x->sys_of, x->sys_box);
    int rc = bh::launch_walk(x->pos_s, x->vals, x->g_first, x->g_count, x->nd, x->cfg.order, x->cfg.group_size, eps,
                             (float4*)d_acc_pot, x->ctrl, x->sm_count, x->cfg.block_threads, x->cfg.blocks_per_sm, s,
                             nullptr, x->cfg.walk_variant);
    if (rc) return rc;
    // init, batch sort, 4 tree, 5 groups, moments per level, 2 walk
    x->launches += 2 + 4 + 5 + bh::launches_moments(x->deep) + bh::kLaunchesForce;
    if (cudaGetLastError() != cudaSuccess) return BH_ERR_CUDA;
    x->n = n;
    x->theta = theta;
    x->have_moments = false;  // the tree of several systems is not for tree_force
    return BH_OK;
}

int bh_graph_capture_batched(bh_ctx* x, const float* d_pos_mass, float theta, float eps, float* d_acc_pot,
                             void** graph_exec)
{
    if (!x || !graph_exec) return BH_ERR_INVALID;
    *graph_exec = nullptr;
    DeviceGuard guard(x->device);
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return BH_ERR_CUDA;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return BH_ERR_CUDA;
    }
    const int rc = bh_force_batched(x, d_pos_mass, theta, eps, d_acc_pot, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != BH_OK || ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != BH_OK ? rc : BH_ERR_CUDA;
    }
    cudaGraphExec_t ge = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return BH_ERR_CUDA;
    }
    *graph_exec = (void*)ge;
    return BH_OK;
}

int bh_graph_launch(void* graph_exec, void* stream)
{
    if (!graph_exec) return BH_ERR_INVALID;
    return cudaGraphLaunch((cudaGraphExec_t)graph_exec, (cudaStream_t)stream) == cudaSuccess ? BH_OK : BH_ERR_CUDA;
}

void bh_graph_destroy(void* graph_exec)
{
    if (graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)graph_exec);
}

}  // extern "C"

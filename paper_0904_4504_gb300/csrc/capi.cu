// capi.cu -- host runtime and C ABI of liblbm.so (declarations and contracts in include/lbm.h).
//
// The runtime rasterizes the geometry, classifies nodes and blocked links once, owns the device
// buffers of a simulation, tabulates the drive in FP64, launches the fused step kernel once per
// time step on the simulation's stream, and reads back the FP64 force history.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm.h"
#include "runtime.h"
#include "pbatch.cuh"

namespace lbm {

void* find_tma_launcher_q9(int storage, int coll, int variant);
void* find_q9v_launcher(int storage, int coll, int variant);
void tma_box_q9(int storage, int bx, int* bw, int* pad);

// D2Q37 launch tables, one translation unit per storage type (step_q37_inst.cuh).
#define LBM_Q37_DECLS(SFX)                                          \
    void* find_launcher_q37_##SFX(int coll);                        \
    PbKernel find_pbatch_q37_##SFX(int coll, int variant);          \
    void* find_launcher_q37_##SFX##_ds(int coll);                   \
    void* find_occ_launcher_q37_##SFX(int coll, int variant);       \
    void* find_tma_launcher_q37_##SFX(int coll, int variant);       \
    void tma_box_q37_##SFX(int bx, int* bw, int* pad);
LBM_Q37_DECLS(f64)
LBM_Q37_DECLS(f32)
LBM_Q37_DECLS(bf16)
LBM_Q37_DECLS(f16)
#undef LBM_Q37_DECLS

struct Q37Table {
    void* (*plain)(int coll);
    PbKernel (*pbatch)(int coll, int variant);
    void* (*plain_ds)(int coll);
    void* (*occ)(int coll, int variant);
    void* (*tma)(int coll, int variant);
    void (*box)(int bx, int* bw, int* pad);
};

static const Q37Table* q37_table(int storage) {
#define LBM_Q37_ROW(SFX)                                                                          \
    {find_launcher_q37_##SFX, find_pbatch_q37_##SFX, find_launcher_q37_##SFX##_ds, find_occ_launcher_q37_##SFX, \
     find_tma_launcher_q37_##SFX, tma_box_q37_##SFX}
    static const Q37Table rows[4] = {LBM_Q37_ROW(f64), LBM_Q37_ROW(f32), LBM_Q37_ROW(bf16), LBM_Q37_ROW(f16)};
#undef LBM_Q37_ROW
    return storage >= ST_F64 && storage <= ST_F16 ? &rows[storage] : nullptr;
}

static TmaStepLaunchFn find_tma_launcher(int Q, int storage, int coll, int variant) {
    void* f = nullptr;
    if (Q == 9) f = find_tma_launcher_q9(storage, coll, variant);
    else if (Q == 37 && q37_table(storage)) f = q37_table(storage)->tma(coll, variant);
    return reinterpret_cast<TmaStepLaunchFn>(f);
}

// Tile of a staged variant (see lbm_set_variant); false for other variants.
static bool variant_tile(int variant, int* bx, int* by) {
    switch (variant) {
        case 1:
        case 2:
        case 10: *bx = 32; *by = 4; return true;
        case 3: *bx = 32; *by = 8; return true;
        case 4: *bx = 32; *by = 16; return true;
        case 11: *bx = 64; *by = 2; return true;
        case 12: *bx = 64; *by = 4; return true;
        case 13: *bx = 64; *by = 2; return true;
        case 18: *bx = 64; *by = 4; return true;
        case 23: *bx = 64; *by = 2; return true;
        case 24: *bx = 64; *by = 4; return true;
        case 25: *bx = 128; *by = 2; return true;
        case 26:
        case 27: *bx = 64; *by = 3; return true;
        case 28: *bx = 128; *by = 3; return true;
        case 20: *bx = 64; *by = 4; return true;
        case 30: *bx = 128; *by = 4; return true;
        case 21: *bx = 64; *by = 2; return true;
        case 22: *bx = 128; *by = 2; return true;
        default: return false;
    }
}

static void tma_box(int Q, int storage, int bx, int* bw, int* pad) {
    *bw = *pad = 0;
    if (Q == 9) tma_box_q9(storage, bx, bw, pad);
    else if (Q == 37 && q37_table(storage)) q37_table(storage)->box(bx, bw, pad);
}

// Tensor map of one population buffer: 3-D (x, y, direction), boxes of bw x by x 1.
static int encode_map(CUtensorMap* map, void* base, int storage, int nx, int ny, int Q, int pitch, int bw, int by) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return set_error(LBM_ECUDA, "cuTensorMapEncodeTiled is not available");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const size_t es = storage_size(storage);
    CUtensorMapDataType dt = storage == ST_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : storage == ST_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                             : storage == ST_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)Q};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)pitch * es * ny};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(LBM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LBM_OK;
}

void* find_launcher_q9(int storage, int coll);
void* find_launcher_q9_ds(int storage, int coll);
PbKernel find_pbatch_q9(int storage, int coll, int variant);

static void* find_launcher(int Q, int storage, int coll) {
    if (Q == 9) return find_launcher_q9(storage, coll);
    if (Q == 37 && q37_table(storage)) return q37_table(storage)->plain(coll);
    return nullptr;
}

StepLaunchFn find_occ_launcher(int Q, int storage, int coll, int variant) {
    if (Q != 37 || variant < 1 || variant > 4 || !q37_table(storage)) return nullptr;
    return reinterpret_cast<StepLaunchFn>(q37_table(storage)->occ(coll, variant));
}

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("LBM_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

StepLaunchFn find_aa_launcher_q9(int storage, int coll, int phase);
StepLaunchFn find_aa_launcher_q37_wide(int storage, int coll, int phase);
StepLaunchFn find_aa_launcher_q37_half(int storage, int coll, int phase);

StepLaunchFn find_aa_launcher(int Q, int storage, int coll, int phase) {
    if (Q == 9) return find_aa_launcher_q9(storage, coll, phase);
    if (Q == 37) return storage <= ST_F32 ? find_aa_launcher_q37_wide(storage, coll, phase)
                                          : find_aa_launcher_q37_half(storage, coll, phase);
    return nullptr;
}

StepLaunchFn find_step_launcher(int Q, int storage, int coll, int wall) {
    if (wall == 0) return reinterpret_cast<StepLaunchFn>(find_launcher(Q, storage, coll));
    void* f = nullptr;
    if (Q == 9) f = find_launcher_q9_ds(storage, coll);
    else if (Q == 37 && q37_table(storage)) f = q37_table(storage)->plain_ds(coll);
    return reinterpret_cast<StepLaunchFn>(f);
}
PbKernel find_pbatch_kernel(int Q, int storage, int coll, int variant) {
    if (Q == 9) return find_pbatch_q9(storage, coll, variant);
    if (Q == 37 && q37_table(storage)) return q37_table(storage)->pbatch(coll, variant);
    return PbKernel{nullptr, dim3(), 0, 0, 0};
}

// ---------------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------------

static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

void clear_error() { g_err.clear(); }

const char* last_error() { return g_err.c_str(); }

// ---------------------------------------------------------------------------------------------
// lattice tables on the host (same constants as the device, lattice.cuh)
// ---------------------------------------------------------------------------------------------

template <class L>
static void fill_lattice(HostLattice& H) {
    H.Q = L::Q;
    H.R = L::R;
    H.theta = L::theta();
    for (int i = 0; i < L::Q; ++i) {
        H.c[i][0] = cx_of<L>(i);
        H.c[i][1] = cy_of<L>(i);
        H.w[i] = w_of<L>(i);
        H.opp[i] = opp_of<L>(i);
    }
}

bool host_lattice(int Q, HostLattice& H) {
    if (Q == 9) { fill_lattice<D2Q9>(H); return true; }
    if (Q == 37) { fill_lattice<D2Q37>(H); return true; }
    return false;
}

size_t storage_size(int storage) {
    switch (storage) {
        case ST_F64: return 8;
        case ST_F32: return 4;
        case ST_BF16:
        case ST_F16: return 2;
        default: return 0;
    }
}

// ---------------------------------------------------------------------------------------------
// geometry: labels, node classes and blocked links
// ---------------------------------------------------------------------------------------------

int build_labels(int Q, int nx, int ny, const lbm_geometry& g, std::vector<uint8_t>& lab) {
    HostLattice H;
    host_lattice(Q, H);
    lab.assign((size_t)nx * ny, 0);
    switch (g.kind) {
        case LBM_GEOM_NONE:
            break;
        case LBM_GEOM_PLATE:
            if (ny < 2 * H.R + 1) return set_error(LBM_EINVAL, "plate needs ny >= %d", 2 * H.R + 1);
            for (int y = 0; y < H.R; ++y)
                for (int x = 0; x < nx; ++x) {
                    lab[(size_t)y * nx + x] = LBM_BODY;
                    lab[(size_t)(ny - 1 - y) * nx + x] = LBM_WALL;
                }
            break;
        case LBM_GEOM_BEAM: {
            if (g.lx < 1 || g.ly < 1 || g.lx > nx - 2 * H.R || g.ly > ny - 2 * H.R)
                return set_error(LBM_EINVAL, "beam %dx%d does not fit a %dx%d box with a %d-node gap", g.lx, g.ly,
                                 nx, ny, H.R);
            const int x0 = (nx - g.lx) / 2, y0 = (ny - g.ly) / 2;
            for (int y = y0; y < y0 + g.ly; ++y)
                for (int x = x0; x < x0 + g.lx; ++x) lab[(size_t)y * nx + x] = LBM_BODY;
            break;
        }
        case LBM_GEOM_MASK:
            if (!g.mask) return set_error(LBM_EINVAL, "LBM_GEOM_MASK needs a mask");
            for (size_t k = 0; k < lab.size(); ++k) {
                if (g.mask[k] > LBM_WALL) return set_error(LBM_EINVAL, "mask label %d at %zu", g.mask[k], k);
                lab[k] = g.mask[k];
            }
            break;
        default:
            return set_error(LBM_EINVAL, "unknown geometry kind %d", g.kind);
    }
    return LBM_OK;
}

static int gcd_int(int a, int b) {
    while (b) {
        const int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// For every fluid node, the links whose pull source, or a lattice node strictly between source and
// node, is solid; the first solid node met walking back from the node decides body or wall.  Only
// rows within R of a row holding a solid node can have solid or boundary nodes; the others are bulk
// fluid and are not visited (a large domain around a small body is mostly such rows).  `links`
// lists the boundary nodes in increasing node order.
void build_links(const HostLattice& H, int nx, int ny, const std::vector<uint8_t>& lab, std::vector<uint8_t>& cls,
                 std::vector<LinkNode>& links, size_t& n_fluid) {
    const size_t N = (size_t)nx * ny;
    cls.assign(N, NODE_BULK);
    links.clear();
    auto wrap = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };  // nx, ny > R
    // solid within R along x of each node of the rows holding a solid, scattered from the solids
    std::vector<uint8_t> rowsolid(ny, 0), rownear(N, 0), near(nx);
    size_t n_solid = 0;
    for (int y = 0; y < ny; ++y) {
        const uint8_t* L = lab.data() + (size_t)y * nx;
        uint8_t* O = rownear.data() + (size_t)y * nx;
        for (int x = 0; x < nx; ++x) {
            if (!L[x]) continue;
            rowsolid[y] = 1;
            ++n_solid;
            for (int d = -H.R; d <= H.R; ++d) O[wrap(x + d, nx)] = 1;
        }
    }
    n_fluid = N - n_solid;
    for (int y = 0; y < ny; ++y) {
        // solid within R of each node of row y: the rows within R along y or-ed together
        bool any = false;
        for (int d = -H.R; d <= H.R; ++d) any = any || rowsolid[wrap(y + d, ny)];
        if (!any) continue;
        std::fill(near.begin(), near.end(), 0);
        for (int d = -H.R; d <= H.R; ++d) {
            const int ys = wrap(y + d, ny);
            if (!rowsolid[ys]) continue;
            const uint8_t* I = rownear.data() + (size_t)ys * nx;
            for (int x = 0; x < nx; ++x) near[x] |= I[x];
        }
        for (int x = 0; x < nx; ++x) {
            const size_t node = (size_t)y * nx + x;
            if (lab[node]) {
                cls[node] = NODE_SOLID;
                continue;
            }
            if (!near[x]) continue;
            uint64_t b = 0, w = 0;
            for (int i = 1; i < H.Q; ++i) {
                const int cx = H.c[i][0], cy = H.c[i][1];
                const int g = gcd_int(std::abs(cx), std::abs(cy));
                for (int k = 1; k <= g; ++k) {
                    const int sx = wrap(x - k * cx / g, nx);
                    const int sy = wrap(y - k * cy / g, ny);
                    const uint8_t l = lab[(size_t)sy * nx + sx];
                    if (l) {
                        (l == LBM_BODY ? b : w) |= 1ull << i;
                        break;
                    }
                }
            }
            if (b | w) {
                cls[node] = NODE_BOUNDARY;
                links.push_back(LinkNode{node, b, w});
            }
        }
    }
}

// Geometry-only part of the momentum exchange (the rest populations w_i rho0 bounced on body
// links): -sum over body links of c_i 2 w_i rho0.
void constant_force(const HostLattice& H, const std::vector<LinkNode>& links, double rho0, double& fx, double& fy) {
    fx = fy = 0.0;
    for (const LinkNode& ln : links) {
        const uint64_t b = ln.body;
        if (!b) continue;
        for (int i = 1; i < H.Q; ++i)
            if ((b >> i) & 1ull) {
                fx -= H.c[i][0] * 2.0 * H.w[i] * rho0;
                fy -= H.c[i][1] * 2.0 * H.w[i] * rho0;
            }
    }
}

void tile_slots(int nx, int ny, int bx, int by, const std::vector<LinkNode>& links, std::vector<int>& slot, int& ntx,
                int& ntiles, int& nslots) {
    ntx = (nx + bx - 1) / bx;
    const int nty = (ny + by - 1) / by;
    ntiles = ntx * nty;
    slot.assign(ntiles, -1);
    for (const LinkNode& ln : links) {
        if (!ln.body) continue;
        const int x = (int)(ln.node % (size_t)nx), y = (int)(ln.node / (size_t)nx);
        slot[(y / by) * ntx + x / bx] = 0;  // tile with body links
    }
    nslots = 0;
    for (int t = 0; t < ntiles; ++t)
        if (slot[t] == 0) slot[t] = nslots++;
}

double drive_value(int drive, double u0, double omega, long n) {
    const double t = (double)n + 0.5;
    return drive == LBM_DRIVE_WALL ? u0 * std::sin(omega * t) : u0 * omega * std::cos(omega * t);
}

// ---------------------------------------------------------------------------------------------
// fit (FP64 least squares on {sin, cos, 1})
// ---------------------------------------------------------------------------------------------

int fit_sincos(const double* fx, size_t stride, long n0, long n1, double omega, double coef[3]) {
    double M[3][4] = {{0}};
    for (long n = n0; n < n1; ++n) {
        const double t = (double)n + 0.5;
        const double b[3] = {std::sin(omega * t), std::cos(omega * t), 1.0};
        const double y = fx[(size_t)n * stride];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) M[r][c] += b[r] * b[c];
            M[r][3] += b[r] * y;
        }
    }
    for (int c = 0; c < 3; ++c) {  // Gaussian elimination with partial pivoting
        int p = c;
        for (int r = c + 1; r < 3; ++r)
            if (std::fabs(M[r][c]) > std::fabs(M[p][c])) p = r;
        if (std::fabs(M[p][c]) < 1e-300) return set_error(LBM_ERANGE, "fit window too short");
        if (p != c)
            for (int k = 0; k < 4; ++k) std::swap(M[p][k], M[c][k]);
        for (int r = 0; r < 3; ++r) {
            if (r == c) continue;
            const double f = M[r][c] / M[c][c];
            for (int k = c; k < 4; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < 3; ++r) coef[r] = M[r][3] / M[r][r];
    return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

// ---------------------------------------------------------------------------------------------
// the simulation object
// ---------------------------------------------------------------------------------------------

struct lbm_sim {
    int device = 0;
    int Q = 0, nx = 0, ny = 0, pitch = 0;
    double tau = 0, omega = 0;
    lbm_geometry geom{};
    HostLattice lat{};
    size_t esize = 0;
    std::vector<uint8_t> labels;
    std::vector<LinkNode> link_nodes;  // boundary nodes and their link masks
    size_t n_fluid = 0, n_boundary = 0;
    double fconst[2] = {0, 0};
    // device memory
    void* buf[2] = {nullptr, nullptr};
    uint8_t* d_cls = nullptr;
    ulonglong2* d_links = nullptr;
    int* d_tile_slot = nullptr;
    double2* d_partials = nullptr;
    unsigned int* d_ticket = nullptr;
    int* d_err = nullptr;
    double2* d_history = nullptr;
    size_t cap = 0;
    size_t device_bytes = 0;
    size_t h2d_bytes = 0, d2h_bytes = 0;  // host<->device traffic over the simulation's life
    // state
    long steps_done = 0;
    int cur = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int bx = 32, by = 4, ntx = 0, ntiles = 0, nslots = 0;
    int plain_bx = 32, plain_by = 4;   // tile of the plain kernel (lbm_set_tile)
    int variant = 0;                   // 0 plain kernel, else a staged variant (lbm_set_variant)
    bool stream_off = false;           // 16-bit body frame: store h - H(U(n)), see InstDev
    double U_stream = 0.0;             // U(n) = sum_{k<n} g(k + 1/2) for n = steps_done
    StepLaunchFn launch = nullptr;     // plain step in use (variant 0, or an occupancy variant 1-2)
    StepLaunchFn launch_default = nullptr;
    TmaStepLaunchFn tma_launch = nullptr;
    bool aa = false;                   // in-place single buffer (LBM_LAYOUT_AA)
    StepLaunchFn aa_launch[2] = {nullptr, nullptr};  // even (pull-push) and odd (local) steps
    CUtensorMap maps[2];               // staged variants: load boxes of buffer k
    CUtensorMap store_maps[2];         // variants 13, 14: the tile's own box in buffer k
    InstDev dev{};
};

namespace {

#define CUDA_TRY(expr)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            return set_error(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", \
                             #expr, cudaGetErrorString(e_));                                     \
        }                                                                                        \
    } while (0)

template <class T>
int dev_alloc(lbm_sim* s, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    CUDA_TRY(cudaMalloc((void**)p, count * sizeof(T)));
    s->device_bytes += count * sizeof(T);
    return LBM_OK;
}

void free_sim(lbm_sim* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->buf[0]);
    cudaFree(s->buf[1]);
    cudaFree(s->d_cls);
    cudaFree(s->d_links);
    cudaFree(s->d_tile_slot);
    cudaFree(s->d_partials);
    cudaFree(s->d_ticket);
    cudaFree(s->d_err);
    cudaFree(s->d_history);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

// (Re)build the per-tile force slots for the current tile shape.
int setup_tiles(lbm_sim* s) {
    std::vector<int> slot;
    tile_slots(s->nx, s->ny, s->bx, s->by, s->link_nodes, slot, s->ntx, s->ntiles, s->nslots);
    cudaFree(s->d_tile_slot);
    cudaFree(s->d_partials);
    s->d_tile_slot = nullptr;
    s->d_partials = nullptr;
    int rc = dev_alloc(s, &s->d_tile_slot, slot.size());
    if (rc) return rc;
    // two force partials per slot: the in-place even step records the forces of two steps
    const size_t np = 2 * (size_t)std::max(1, s->nslots);
    rc = dev_alloc(s, &s->d_partials, np);
    if (rc) return rc;
    CUDA_TRY(cudaMemcpy(s->d_tile_slot, slot.data(), slot.size() * sizeof(int), cudaMemcpyHostToDevice));
    s->h2d_bytes += slot.size() * sizeof(int);
    CUDA_TRY(cudaMemset(s->d_partials, 0, np * sizeof(double2)));
    s->dev.tile_slot = s->d_tile_slot;
    s->dev.partials = s->d_partials;
    s->dev.ntx = s->ntx;
    s->dev.ntiles = s->ntiles;
    s->dev.nslots = s->nslots;
    return LBM_OK;
}

// Make room for the force history of `need` steps.
int ensure_capacity(lbm_sim* s, size_t need) {
    if (need <= s->cap) return LBM_OK;
    size_t cap = std::max<size_t>(std::max<size_t>(need, 2 * s->cap), 1024);
    double2* hist = nullptr;
    CUDA_TRY(cudaMalloc((void**)&hist, cap * sizeof(double2)));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    CUDA_TRY(cudaMemset(hist, 0, cap * sizeof(double2)));
    // an in-place even step has already written the force of the step after it
    const size_t keep = std::min(s->cap, (size_t)s->steps_done + (s->aa ? 1 : 0));
    if (s->d_history && keep > 0)
        CUDA_TRY(cudaMemcpy(hist, s->d_history, keep * sizeof(double2), cudaMemcpyDeviceToDevice));
    cudaFree(s->d_history);
    s->device_bytes += (cap - s->cap) * sizeof(double2);
    s->d_history = hist;
    s->cap = cap;
    return LBM_OK;
}

// Scaled equilibrium deviation H_i of the uniform stream U x (no rest term), and its moments.
void stream_offset(const lbm_sim* s, double U, float* H, float* HM) {
    const HostLattice& L = s->lat;
    const double b = U * U / L.theta;
    double M[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < L.Q; ++i) {
        const double a = L.c[i][0] * U / L.theta;
        double poly = a + 0.5 * (a * a - b);
        if (s->geom.eq_order >= 4) poly += (a * a * a - 3 * a * b) / 6.0 + (a * a * a * a - 6 * a * a * b + 3 * b * b) / 24.0;
        const double Hi = s->geom.rho0 * poly / s->dev.s;
        H[i] = (float)Hi;
        const double w = L.w[i], cx = L.c[i][0], cy = L.c[i][1];
        M[0] += w * H[i];
        M[1] += w * cx * H[i];
        M[2] += w * cy * H[i];
        M[3] += w * cx * cx * H[i];
        M[4] += w * cx * cy * H[i];
        M[5] += w * cy * cy * H[i];
    }
    if (HM)
        for (int k = 0; k < 6; ++k) HM[k] = (float)M[k];
}

// The same constants for the kernels: H_i depends on c_ix only, so they get it per c_ix (index
// c_ix + 3), and the moments HM.
void stream_offset_cx(const lbm_sim* s, double U, float* H7, float* HM) {
    float H[37];
    stream_offset(s, U, H, HM);
    for (int k = 0; k < 7; ++k) H7[k] = 0.f;
    for (int i = 0; i < s->lat.Q; ++i) H7[s->lat.c[i][0] + 3] = H[i];
}

// Even and odd parts in c_x of the stored state's offsets, for m = |c_x| (see InstDev).
void stream_offset_eo(const float* H7, float* He, float* Ho) {
    for (int m = 0; m < 4; ++m) {
        He[m] = 0.5f * (H7[3 + m] + H7[3 - m]);
        Ho[m] = 0.5f * (H7[3 + m] - H7[3 - m]);
    }
}

int check_sim(lbm_sim* s) {
    if (!s) return set_error(LBM_EINVAL, "null simulation");
    CUDA_TRY(cudaSetDevice(s->device));
    return LBM_OK;
}

}  // namespace

namespace lbm {

// Read-only view of a simulation for other translation units of the library.
SimView sim_view(const lbm_sim* s) {
    SimView v;
    v.device = s->device;
    v.Q = s->Q;
    v.storage = s->geom.storage;
    v.collision = s->geom.collision;
    v.nx = s->nx;
    v.ny = s->ny;
    v.pitch = s->pitch;
    v.bx = s->bx;
    v.by = s->by;
    v.nslots = s->nslots;
    v.drive = s->geom.drive;
    v.u0 = s->geom.u0;
    v.omega = s->omega;
    v.inst = s->dev;
    v.buf[0] = s->buf[0];
    v.buf[1] = s->buf[1];
    v.cur = s->cur;
    v.steps_done = s->steps_done;
    v.history = s->d_history;
    v.esize = s->esize;
    v.n_fluid = s->n_fluid;
    v.aa = s->aa ? 1 : 0;
    v.variant = s->variant;
    v.ntiles = s->ntiles;
    v.maps = s->maps;
    return v;
}

int sim_reserve(lbm_sim* s, size_t steps) { return ensure_capacity(s, steps); }

void sim_disable_stream_offset(lbm_sim* s) {
    if (s->steps_done == 0) s->stream_off = false;
    s->dev.stream_off = s->stream_off ? 1 : 0;
}

void sim_advance(lbm_sim* s, long steps) {
    if (s->stream_off)
        for (long k = 0; k < steps; ++k) s->U_stream += drive_value(s->geom.drive, s->geom.u0, s->omega, s->steps_done + k);
    s->steps_done += steps;
    s->cur ^= (int)(steps & 1);
}

void sim_step_constants(const lbm_sim* s, long count, StepConst* out) {
    double U = s->U_stream;
    for (long k = 0; k < count; ++k) {
        StepConst& c = out[k];
        std::memset(&c, 0, sizeof(c));
        c.dv = drive_value(s->geom.drive, s->geom.u0, s->omega, s->steps_done + k);
        c.dv_f = (float)c.dv;
        if (s->stream_off) {
            float* H = c.H;  // HM[6], Hl[7], Hs[7], He[4], Ho[4]
            stream_offset_cx(s, U, H + 6, H);
            stream_offset_cx(s, U + c.dv, H + 13, nullptr);
            stream_offset_eo(H + 13, H + 20, H + 24);
            U += c.dv;
        }
    }
}

}  // namespace lbm

extern "C" {

const char* lbm_last_error(void) { return last_error(); }

int lbm_geometry_links(int lattice, int nx, int ny, const lbm_geometry* geom, unsigned char* cls,
                       unsigned long long* body, unsigned long long* wall, size_t count, size_t* n_fluid,
                       size_t* n_boundary) {
    clear_error();
    HostLattice H;
    if (!host_lattice(lattice, H)) return set_error(LBM_EINVAL, "unknown lattice %d", lattice);
    if (!geom) return set_error(LBM_EINVAL, "null geometry");
    if (nx < 2 * H.R + 1 || ny < 2 * H.R + 1)
        return set_error(LBM_EINVAL, "grid %dx%d below %d nodes per side", nx, ny, 2 * H.R + 1);
    if ((long long)nx * ny > (1ll << 31) / 2) return set_error(LBM_EINVAL, "grid %dx%d too large", nx, ny);
    const size_t N = (size_t)nx * ny;
    if ((cls || body || wall) && count < N) return set_error(LBM_EINVAL, "outputs hold %zu < %zu nodes", count, N);
    std::vector<uint8_t> lab, c;
    std::vector<LinkNode> links;
    size_t nf = 0;
    int rc = build_labels(lattice, nx, ny, *geom, lab);
    if (rc) return rc;
    build_links(H, nx, ny, lab, c, links, nf);
    if (cls) std::copy(c.begin(), c.end(), cls);
    if (body) std::fill(body, body + N, 0ull);
    if (wall) std::fill(wall, wall + N, 0ull);
    for (const LinkNode& ln : links) {
        if (body) body[ln.node] = ln.body;
        if (wall) wall[ln.node] = ln.wall;
    }
    if (n_fluid) *n_fluid = nf;
    if (n_boundary) *n_boundary = links.size();
    return LBM_OK;
}

int lbm_lattice_velocities(int lattice, int* c_xy, double* w, double* theta) {
    HostLattice H;
    if (!host_lattice(lattice, H)) return set_error(LBM_EINVAL, "unknown lattice %d", lattice);
    for (int i = 0; i < H.Q; ++i) {
        if (c_xy) { c_xy[2 * i] = H.c[i][0]; c_xy[2 * i + 1] = H.c[i][1]; }
        if (w) w[i] = H.w[i];
    }
    if (theta) *theta = H.theta;
    return H.Q;
}

int lbm_params_from_tau_omega(int lattice, double tau_omega, double delta_min, int p_min, double* tau,
                              double* omega, int* period) {
    HostLattice H;
    if (!host_lattice(lattice, H)) return set_error(LBM_EINVAL, "unknown lattice %d", lattice);
    if (!(tau_omega > 0.0) || !(delta_min > 0.0) || p_min < 1)
        return set_error(LBM_EINVAL, "need tau_omega > 0, delta_min > 0, p_min >= 1");
    const double pi = 3.14159265358979323846;
    const double need = std::ceil(2.0 * pi * delta_min / std::sqrt(2.0 * H.theta * tau_omega));
    if (!(need < 2e9)) return set_error(LBM_EINVAL, "tau_omega %g needs too many steps per period", tau_omega);
    const int P = std::max(p_min, (int)need);
    const double om = 2.0 * pi / P;
    if (tau) *tau = 0.5 + tau_omega / om;
    if (omega) *omega = om;
    if (period) *period = P;
    return LBM_OK;
}

int lbm_create(int lattice, int nx, int ny, double tau, double omega, const lbm_geometry* geom, lbm_sim** out) {
    clear_error();
    if (!out) return set_error(LBM_EINVAL, "null output handle");
    *out = nullptr;
    if (!geom) return set_error(LBM_EINVAL, "null geometry");
    HostLattice H;
    if (!host_lattice(lattice, H)) return set_error(LBM_EINVAL, "lattice must be LBM_D2Q9 or LBM_D2Q37");
    if (nx < 2 * H.R + 1 || ny < 2 * H.R + 1)
        return set_error(LBM_EINVAL, "grid %dx%d below %d nodes per side", nx, ny, 2 * H.R + 1);
    if ((long long)nx * ny > (1ll << 31) / 2) return set_error(LBM_EINVAL, "grid %dx%d too large", nx, ny);
    if (!(tau > 0.5) || !std::isfinite(tau)) return set_error(LBM_EINVAL, "tau must be > 1/2 (got %g)", tau);
    if (!(omega > 0.0) || !std::isfinite(omega)) return set_error(LBM_EINVAL, "omega must be > 0 (got %g)", omega);
    lbm_geometry g = *geom;
    if (g.rho0 == 0.0) g.rho0 = 1.0;
    if (!(g.rho0 > 0.0)) return set_error(LBM_EINVAL, "rho0 must be > 0");
    if (!(g.u0 >= 0.0) || !(g.u0 < omega))
        return set_error(LBM_EINVAL, "need 0 <= u0 < omega (displacement below one node), got u0=%g omega=%g", g.u0,
                         omega);
    if (g.drive != LBM_DRIVE_WALL && g.drive != LBM_DRIVE_BODYFORCE) return set_error(LBM_EINVAL, "bad drive");
    if (g.eq_order != 2 && g.eq_order != 4) return set_error(LBM_EINVAL, "eq_order must be 2 or 4");
    if (lattice == LBM_D2Q9 && g.eq_order != 2) return set_error(LBM_EINVAL, "D2Q9 supports eq_order 2 only");
    if (g.collision != LBM_COLL_BGK && g.collision != LBM_COLL_REGULARIZED)
        return set_error(LBM_EINVAL, "bad collision");
    if (g.wall_scheme != LBM_SCHEME_BOUNCEBACK && g.wall_scheme != LBM_SCHEME_DIFFUSE)
        return set_error(LBM_EINVAL, "bad wall scheme %d", g.wall_scheme);
    if (g.layout != LBM_LAYOUT_AB && g.layout != LBM_LAYOUT_AA) return set_error(LBM_EINVAL, "bad layout %d", g.layout);
    if (g.layout == LBM_LAYOUT_AA && g.wall_scheme != LBM_SCHEME_BOUNCEBACK)
        return set_error(LBM_EINVAL, "the in-place (AA) layout is built for bounce-back walls only");
    const size_t es = storage_size(g.storage);
    if (!es) return set_error(LBM_EINVAL, "bad storage type %d", g.storage);
    if (es == 2 && !(g.u0 > 0.0))
        return set_error(LBM_EINVAL, "16-bit storage is scaled by u0 and needs u0 > 0");
    StepLaunchFn fn = find_step_launcher(lattice, g.storage, g.collision, g.wall_scheme);
    if (!fn) return set_error(LBM_EINVAL, "no kernel for this lattice/storage/collision/wall");
    StepLaunchFn aa0 = nullptr, aa1 = nullptr;
    if (g.layout == LBM_LAYOUT_AA) {
        aa0 = find_aa_launcher(lattice, g.storage, g.collision, 0);
        aa1 = find_aa_launcher(lattice, g.storage, g.collision, 1);
        if (!aa0 || !aa1) return set_error(LBM_EINVAL, "no in-place kernel for this lattice/storage/collision");
    }

    lbm_sim* s = new (std::nothrow) lbm_sim();
    if (!s) return set_error(LBM_ENOMEM, "host allocation");
    s->Q = lattice;
    s->nx = nx;
    s->ny = ny;
    s->tau = tau;
    s->omega = omega;
    s->lat = H;
    s->esize = es;
    s->launch = fn;
    s->launch_default = fn;
    s->aa = g.layout == LBM_LAYOUT_AA;
    s->aa_launch[0] = aa0;
    s->aa_launch[1] = aa1;
    int rc = cudaGetDevice(&s->device) == cudaSuccess ? LBM_OK : LBM_ECUDA;
    if (rc) { delete s; return set_error(rc, "no CUDA device"); }
    rc = build_labels(lattice, nx, ny, g, s->labels);
    if (rc) { delete s; return rc; }
    g.mask = nullptr;
    s->geom = g;
    std::vector<uint8_t> cls;
    build_links(H, nx, ny, s->labels, cls, s->link_nodes, s->n_fluid);
    s->n_boundary = s->link_nodes.size();
    constant_force(H, s->link_nodes, g.rho0, s->fconst[0], s->fconst[1]);

    const int align = (int)(128 / es);
    s->pitch = (nx + align - 1) / align * align;
    const size_t plane = (size_t)ny * s->pitch;
    if ((size_t)H.Q * plane >= (1ull << 32)) {  // the kernels address populations with 32-bit offsets
        delete s;
        return set_error(LBM_EINVAL, "grid %dx%d: %d x %zu populations exceed 2^32", nx, ny, H.Q, plane);
    }

    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return set_error(LBM_ECUDA, "stream creation failed");
    }
    s->own_stream = true;

#define TRY_OR_FREE(x)          \
    do {                        \
        int r_ = (x);           \
        if (r_) {               \
            free_sim(s);        \
            return r_;          \
        }                       \
    } while (0)

    for (int b = 0; b < (s->aa ? 1 : 2); ++b) {
        TRY_OR_FREE(dev_alloc(s, (char**)&s->buf[b], plane * H.Q * es));
        if (cudaMemset(s->buf[b], 0, plane * H.Q * es) != cudaSuccess) {
            free_sim(s);
            return set_error(LBM_ECUDA, "memset");
        }
    }
    // node classes in the padded layout (padding solid); link masks zeroed on the device, then only
    // the rows holding boundary nodes uploaded
    std::vector<uint8_t> cls_p(plane, NODE_SOLID);
    for (int y = 0; y < ny; ++y) std::copy_n(cls.data() + (size_t)y * nx, nx, cls_p.data() + (size_t)y * s->pitch);
    TRY_OR_FREE(dev_alloc(s, &s->d_cls, plane));
    TRY_OR_FREE(dev_alloc(s, &s->d_links, plane));
    TRY_OR_FREE(dev_alloc(s, &s->d_ticket, 1));
    TRY_OR_FREE(dev_alloc(s, &s->d_err, 1));
    bool up = cudaMemcpy(s->d_cls, cls_p.data(), plane, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemset(s->d_links, 0, plane * sizeof(ulonglong2)) == cudaSuccess &&
              cudaMemset(s->d_ticket, 0, sizeof(unsigned)) == cudaSuccess &&
              cudaMemset(s->d_err, 0, sizeof(int)) == cudaSuccess;
    s->h2d_bytes += plane;
    std::vector<ulonglong2> row(s->pitch);
    for (size_t k = 0; up && k < s->link_nodes.size();) {
        const size_t y = s->link_nodes[k].node / (size_t)nx;
        std::fill(row.begin(), row.end(), make_ulonglong2(0, 0));
        for (; k < s->link_nodes.size() && s->link_nodes[k].node / (size_t)nx == y; ++k) {
            const LinkNode& ln = s->link_nodes[k];
            row[ln.node % (size_t)nx] = make_ulonglong2(ln.body, ln.wall);
        }
        up = cudaMemcpy(s->d_links + y * s->pitch, row.data(), s->pitch * sizeof(ulonglong2),
                        cudaMemcpyHostToDevice) == cudaSuccess;
        s->h2d_bytes += s->pitch * sizeof(ulonglong2);
    }
    if (!up) {
        free_sim(s);
        return set_error(LBM_ECUDA, "upload of geometry failed");
    }

    InstDev& d = s->dev;
    d.cls = s->d_cls;
    d.links = s->d_links;
    d.ticket = s->d_ticket;
    d.err = s->d_err;
    d.fconst = make_double2(s->fconst[0], s->fconst[1]);
    d.plane = (long long)plane;
    d.nx = nx;
    d.ny = ny;
    d.pitch = s->pitch;
    d.eq_order = g.eq_order;
    d.moving = g.drive == LBM_DRIVE_WALL;
    d.wall_ds = g.wall_scheme == LBM_SCHEME_DIFFUSE;
    d.body_force = g.drive == LBM_DRIVE_BODYFORCE;
    d.rho0 = g.rho0;
    d.s = es == 2 ? g.u0 : 1.0;
    d.inv_s = 1.0 / d.s;
    d.omega_c = 1.0 / tau;
    d.reg_a = (1.0 - 1.0 / tau) / (2.0 * H.theta * H.theta);
    d.src_k = (1.0 - 0.5 / tau) / H.theta;
    d.mw_k = 2.0 * g.rho0 / (H.theta * d.s);
    d.rho0_f = (float)d.rho0;
    d.s_f = (float)d.s;
    d.inv_s_f = (float)d.inv_s;
    d.omega_c_f = (float)d.omega_c;
    d.reg_a_f = (float)d.reg_a;
    d.src_k_f = (float)d.src_k;
    s->stream_off = es == 2 && g.drive == LBM_DRIVE_BODYFORCE;
    d.stream_off = s->stream_off ? 1 : 0;
    // default kernel: the fastest measured single-instance form -- for D2Q37 the plain kernel with
    // an occupancy floor on the default 32 x 4 tile (variant 1 for FP32, 2 for 16-bit storage), for
    // 16-bit D2Q9 the four-nodes-per-thread kernel on 128 x 4 tiles (variant 30)
    if (!s->aa && g.wall_scheme == LBM_SCHEME_BOUNCEBACK) {
        if (lattice == LBM_D2Q9 && es == 2) {
            StepLaunchFn f = reinterpret_cast<StepLaunchFn>(find_q9v_launcher(g.storage, g.collision, 30));
            if (f) {
                s->launch = f;
                s->variant = 30;
                variant_tile(30, &s->bx, &s->by);
            }
        } else {
            const int v = es == 4 ? 1 : es == 2 ? 2 : 0;
            StepLaunchFn f = v ? find_occ_launcher(lattice, g.storage, g.collision, v) : nullptr;
            if (f) {
                s->launch = f;
                s->variant = v;
            }
        }
    }
    TRY_OR_FREE(setup_tiles(s));
    TRY_OR_FREE(ensure_capacity(s, 1024));
    *out = s;
    return LBM_OK;
}

int lbm_set_tile(lbm_sim* s, int block_x, int block_y) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (block_x < 32 || block_x % 32 || block_y < 1 || block_x * block_y > 512)
        return set_error(LBM_EINVAL, "tile %dx%d: need block_x a multiple of 32 and block_x*block_y <= 512", block_x,
                         block_y);
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    s->plain_bx = s->bx = block_x;
    s->plain_by = s->by = block_y;
    s->variant = 0;
    s->tma_launch = nullptr;
    s->launch = s->launch_default;
    return setup_tiles(s);
}

int lbm_set_variant(lbm_sim* s, int variant) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (variant == 0) return lbm_set_tile(s, s->plain_bx, s->plain_by);
    if (s->aa) return set_error(LBM_EINVAL, "the in-place (AA) layout runs the plain kernel (variant 0) only");
    if (s->geom.wall_scheme != LBM_SCHEME_BOUNCEBACK)
        return set_error(LBM_EINVAL, "kernel variants are built for bounce-back walls only");
    if ((variant >= 1 && variant <= 4) || variant == 30) {
        StepLaunchFn f = variant >= 30 ? (s->Q == 9 ? reinterpret_cast<StepLaunchFn>(find_q9v_launcher(
                                                          s->geom.storage, s->geom.collision, variant))
                                                    : nullptr)
                                       : find_occ_launcher(s->Q, s->geom.storage, s->geom.collision, variant);
        if (!f) return set_error(LBM_EINVAL, "variant %d is not built for this lattice/storage/collision", variant);
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        variant_tile(variant, &s->bx, &s->by);
        s->variant = variant;
        s->tma_launch = nullptr;
        s->launch = f;
        return setup_tiles(s);
    }
    int bx, by, bw, pad;
    TmaStepLaunchFn fn = find_tma_launcher(s->Q, s->geom.storage, s->geom.collision, variant);
    if (!fn || !variant_tile(variant, &bx, &by))
        return set_error(LBM_EINVAL, "variant %d is not built for this lattice/storage/collision", variant);
    tma_box(s->Q, s->geom.storage, bx, &bw, &pad);
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    for (int k = 0; k < 2; ++k) {
        if ((rc = encode_map(&s->maps[k], s->buf[k], s->geom.storage, s->nx, s->ny, s->Q, s->pitch, bw, by)))
            return rc;
        if ((rc = encode_map(&s->store_maps[k], s->buf[k], s->geom.storage, s->nx, s->ny, s->Q, s->pitch, bx, by)))
            return rc;
    }
    s->bx = bx;
    s->by = by;
    s->variant = variant;
    s->tma_launch = fn;
    return setup_tiles(s);
}

int lbm_step(lbm_sim* s, long n) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (n < 0) return set_error(LBM_EINVAL, "negative step count");
    if (n == 0) return LBM_OK;
    // an in-place even step also writes the force of the step after it
    rc = ensure_capacity(s, (size_t)(s->steps_done + n + (s->aa ? 1 : 0)));
    if (rc) return rc;
    const dim3 block(s->bx, s->by);
    if (s->aa) {
        for (long k = 0; k < n; ++k) {
            const int phase = (int)(s->steps_done & 1);
            s->dev.src = s->buf[0];
            s->dev.dst = s->buf[0];
            s->dev.dv = drive_value(s->geom.drive, s->geom.u0, s->omega, s->steps_done);
            s->dev.dv_f = (float)s->dev.dv;
            s->dev.dv2 = drive_value(s->geom.drive, s->geom.u0, s->omega, s->steps_done + 1);
            s->dev.dv2_f = (float)s->dev.dv2;
            s->dev.stream_off = s->stream_off ? 1 : 0;
            if (s->stream_off) {
                stream_offset_cx(s, s->U_stream, s->dev.Hl, s->dev.HM);
                stream_offset_cx(s, s->U_stream + s->dev.dv, s->dev.Hs, nullptr);
                stream_offset_eo(s->dev.Hs, s->dev.He, s->dev.Ho);
            }
            s->dev.force_out = s->d_history + s->steps_done;
            const cudaError_t e = s->aa_launch[phase](s->dev, block, s->stream);
            if (e != cudaSuccess) return set_error(LBM_ECUDA, "step launch: %s", cudaGetErrorString(e));
            ++s->steps_done;
            if (s->stream_off) s->U_stream += s->dev.dv;
        }
        return LBM_OK;
    }
    for (long k = 0; k < n; ++k) {
        s->dev.src = s->buf[s->cur];
        s->dev.dst = s->buf[s->cur ^ 1];
        s->dev.dv = drive_value(s->geom.drive, s->geom.u0, s->omega, s->steps_done);
        s->dev.dv_f = (float)s->dev.dv;
        s->dev.stream_off = s->stream_off ? 1 : 0;
        if (s->stream_off) {
            stream_offset_cx(s, s->U_stream, s->dev.Hl, s->dev.HM);
            stream_offset_cx(s, s->U_stream + s->dev.dv, s->dev.Hs, nullptr);
            stream_offset_eo(s->dev.Hs, s->dev.He, s->dev.Ho);
        }
        s->dev.force_out = s->d_history + s->steps_done;
        const cudaError_t e = s->tma_launch ? s->tma_launch(s->dev, s->maps[s->cur], s->store_maps[s->cur ^ 1], s->stream)
                                            : s->launch(s->dev, block, s->stream);
        if (e != cudaSuccess) return set_error(LBM_ECUDA, "step launch: %s", cudaGetErrorString(e));
        s->cur ^= 1;
        ++s->steps_done;
        if (s->stream_off) s->U_stream += s->dev.dv;
    }
    return LBM_OK;
}

int lbm_synchronize(lbm_sim* s) {
    int rc = check_sim(s);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    int err = 0;
    CUDA_TRY(cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & 4) return set_error(LBM_ETIMEOUT, "a bounded wait for staged tile loads timed out");
    if (err & 1) return set_error(LBM_ENONFINITE, "force became non-finite: the run diverged");
    return LBM_OK;
}

int lbm_force_history(lbm_sim* s, double* out_xy, size_t cap_steps, size_t* n_steps) {
    int rc = lbm_synchronize(s);
    if (rc && rc != LBM_ENONFINITE) return rc;
    if (n_steps) *n_steps = (size_t)s->steps_done;
    const size_t n = std::min(cap_steps, (size_t)s->steps_done);
    if (n && !out_xy) return set_error(LBM_EINVAL, "null output buffer");
    if (n) CUDA_TRY(cudaMemcpy(out_xy, s->d_history, n * sizeof(double2), cudaMemcpyDeviceToHost));
    s->d2h_bytes += n * sizeof(double2);
    return rc;
}

int lbm_fit(lbm_sim* s, double skip_periods, double* f_in, double* f_q, double* f_0) {
    int rc = check_sim(s);
    if (rc) return rc;
    const double pi = 3.14159265358979323846;
    const double period = 2.0 * pi / s->omega;
    if (!(skip_periods >= 0.0)) return set_error(LBM_EINVAL, "skip_periods must be >= 0");
    const long n0 = (long)std::ceil(skip_periods * period);
    if ((double)(s->steps_done - n0) < period) return set_error(LBM_ERANGE, "less than one period after the skip");
    std::vector<double> h(2 * (size_t)s->steps_done);
    size_t n = 0;
    rc = lbm_force_history(s, h.data(), (size_t)s->steps_done, &n);
    if (rc) return rc;
    double coef[3];
    rc = fit_sincos(h.data(), 2, n0, s->steps_done, s->omega, coef);
    if (rc) return rc;
    const double sgn = s->geom.drive == LBM_DRIVE_WALL ? 1.0 : -1.0;
    if (f_in) *f_in = sgn * coef[0];
    if (f_q) *f_q = sgn * coef[1];
    if (f_0) *f_0 = coef[2];
    return LBM_OK;
}

int lbm_gamma_bar(lbm_sim* s, double f_in, double perimeter, double* gamma_bar) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!gamma_bar || !(perimeter > 0.0) || !(s->geom.u0 > 0.0))
        return set_error(LBM_EINVAL, "need an output, perimeter > 0 and u0 > 0");
    *gamma_bar = -f_in / (s->geom.u0 * s->geom.rho0 * std::sqrt(s->lat.theta / 2.0) * perimeter);
    return LBM_OK;
}

void lbm_destroy(lbm_sim* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    free_sim(s);
}

int lbm_set_stream(lbm_sim* s, void* stream) {
    int rc = check_sim(s);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (s->own_stream) cudaStreamDestroy(s->stream);
    s->stream = (cudaStream_t)stream;
    s->own_stream = false;
    return LBM_OK;
}

static double to_double(const void* base, int storage, size_t k) {
    switch (storage) {
        case ST_F64: return static_cast<const double*>(base)[k];
        case ST_F32: return static_cast<const float*>(base)[k];
        case ST_BF16: return (double)__bfloat162float(static_cast<const __nv_bfloat16*>(base)[k]);
        default: return (double)__half2float(static_cast<const __half*>(base)[k]);
    }
}

static void from_double(void* base, int storage, size_t k, double v) {
    switch (storage) {
        case ST_F64: static_cast<double*>(base)[k] = v; break;
        case ST_F32: static_cast<float*>(base)[k] = (float)v; break;
        case ST_BF16: static_cast<__nv_bfloat16*>(base)[k] = __double2bfloat16(v); break;
        default: static_cast<__half*>(base)[k] = __double2half(v); break;
    }
}

int lbm_get_state(lbm_sim* s, double* out, size_t count) {
    int rc = lbm_synchronize(s);
    if (rc && rc != LBM_ENONFINITE) return rc;
    const size_t N = (size_t)s->nx * s->ny, plane = (size_t)s->ny * s->pitch;
    if (!out || count != N * s->Q) return set_error(LBM_ERANGE, "need %zu values", N * s->Q);
    if (s->aa && (s->steps_done & 1))
        return set_error(LBM_ERANGE, "the in-place layout holds the state after an even number of steps only");
    std::vector<unsigned char> host(plane * s->Q * s->esize);
    CUDA_TRY(cudaMemcpy(host.data(), s->buf[s->cur], host.size(), cudaMemcpyDeviceToHost));
    float H[37] = {0};
    if (s->stream_off) stream_offset(s, s->U_stream, H, nullptr);
    for (int i = 0; i < s->Q; ++i) {
        const double scale = s->lat.w[i] * s->dev.s;
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                const size_t k = (size_t)y * s->nx + x;
                // in place, after an even step count direction i sits in plane opp(i)
                const int pi = s->aa ? s->lat.opp[i] : i;
                const double v = to_double(host.data(), s->geom.storage, (size_t)pi * plane + (size_t)y * s->pitch + x);
                // with the stream offset the kernel forms h = stored + H in FP32; do the same here
                const double h = s->stream_off ? (double)(float)(v + H[i]) : v;
                out[(size_t)i * N + k] = s->labels[k] ? 0.0 : scale * h;
            }
    }
    return rc;
}

int lbm_set_state(lbm_sim* s, const double* g, size_t count) {
    int rc = lbm_synchronize(s);
    if (rc) return rc;
    const size_t N = (size_t)s->nx * s->ny, plane = (size_t)s->ny * s->pitch;
    if (!g || count != N * s->Q) return set_error(LBM_ERANGE, "need %zu values", N * s->Q);
    if (s->aa && (s->steps_done & 1))
        return set_error(LBM_ERANGE, "the in-place layout takes a state after an even number of steps only");
    std::vector<unsigned char> host(plane * s->Q * s->esize, 0);
    float H[37] = {0};
    if (s->stream_off) stream_offset(s, s->U_stream, H, nullptr);
    for (int i = 0; i < s->Q; ++i) {
        const double inv = 1.0 / (s->lat.w[i] * s->dev.s);
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                const size_t k = (size_t)y * s->nx + x;
                const double v = s->labels[k] ? 0.0 : g[(size_t)i * N + k] * inv - (double)H[i];
                const int pi = s->aa ? s->lat.opp[i] : i;
                from_double(host.data(), s->geom.storage, (size_t)pi * plane + (size_t)y * s->pitch + x, v);
            }
    }
    CUDA_TRY(cudaMemcpy(s->buf[s->cur], host.data(), host.size(), cudaMemcpyHostToDevice));
    return LBM_OK;
}

int lbm_get_labels(lbm_sim* s, unsigned char* out, size_t count) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!out || count != s->labels.size()) return set_error(LBM_ERANGE, "need %zu labels", s->labels.size());
    std::memcpy(out, s->labels.data(), count);
    return LBM_OK;
}

int lbm_tune(lbm_sim* s, int steps, lbm_tune_entry* out, int cap, int* n_out) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (steps < 1 || !n_out || (cap > 0 && !out)) return set_error(LBM_EINVAL, "need steps >= 1 and an output");
    // candidates: plain kernel tiles, then every staged variant built for this storage type
    const int tiles[][2] = {{32, 4}, {32, 8}, {64, 2}, {64, 4}, {128, 1}, {32, 2}};
    const int variants[] = {1, 2, 3, 4, 10, 11, 12, 13, 18, 20, 23, 24, 25, 26, 27};
    std::vector<lbm_tune_entry> cand;
    for (auto& t : tiles) cand.push_back(lbm_tune_entry{0, t[0], t[1], 0.0});
    for (int v : variants)
        if (!s->aa && s->geom.wall_scheme == LBM_SCHEME_BOUNCEBACK &&
            (find_tma_launcher(s->Q, s->geom.storage, s->geom.collision, v) ||
             find_occ_launcher(s->Q, s->geom.storage, s->geom.collision, v))) {
            int bx = 0, by = 0;
            variant_tile(v, &bx, &by);
            cand.push_back(lbm_tune_entry{v, bx, by, 0.0});
        }
    // a clone with the same geometry (as a label mask), parameters and storage
    lbm_geometry g = s->geom;
    g.kind = LBM_GEOM_MASK;
    g.mask = s->labels.data();
    lbm_sim* c = nullptr;
    if ((rc = lbm_create(s->Q, s->nx, s->ny, s->tau, s->omega, &g, &c))) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int k = 0;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = set_error(LBM_ECUDA, "events");
    for (auto& e : cand) {
        if (rc) break;
        rc = e.variant ? lbm_set_variant(c, e.variant) : lbm_set_tile(c, e.block_x, e.block_y);
        if (rc) break;
        if ((rc = lbm_step(c, 2))) break;  // warm-up (first launch sets kernel attributes)
        cudaEventRecord(e0, c->stream);
        if ((rc = lbm_step(c, steps))) break;
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = set_error(LBM_ECUDA, "event sync"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        e.us_per_step = 1000.0 * ms / steps;
        if (k < cap) out[k] = e;
        ++k;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lbm_destroy(c);
    *n_out = k;
    return rc;
}

int lbm_autotune(lbm_sim* s, int steps, lbm_tune_entry* best) {
    lbm_tune_entry e[32];
    int n = 0;
    int rc = lbm_tune(s, steps, e, 32, &n);
    if (rc) return rc;
    if (n == 0) return set_error(LBM_EINVAL, "no candidate");
    int b = 0;
    for (int k = 1; k < n; ++k)
        if (e[k].us_per_step < e[b].us_per_step) b = k;
    rc = e[b].variant ? lbm_set_variant(s, e[b].variant) : lbm_set_tile(s, e[b].block_x, e[b].block_y);
    if (rc == LBM_OK && best) *best = e[b];
    return rc;
}

int lbm_info(lbm_sim* s, lbm_info_t* o) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!o) return set_error(LBM_EINVAL, "null output");
    o->lattice = s->Q;
    o->nx = s->nx;
    o->ny = s->ny;
    o->pitch = s->pitch;
    o->storage = s->geom.storage;
    o->collision = s->geom.collision;
    o->eq_order = s->geom.eq_order;
    o->drive = s->geom.drive;
    o->tau = s->tau;
    o->omega = s->omega;
    o->u0 = s->geom.u0;
    o->rho0 = s->geom.rho0;
    o->theta = s->lat.theta;
    o->steps_done = s->steps_done;
    o->n_fluid = s->n_fluid;
    o->n_boundary = s->n_boundary;
    o->bytes_per_step = 2 * (size_t)s->Q * s->esize * s->n_fluid;
    o->device_bytes = s->device_bytes;
    o->block_x = s->bx;
    o->block_y = s->by;
    o->h2d_bytes = s->h2d_bytes;
    o->d2h_bytes = s->d2h_bytes;
    o->variant = s->variant;
    o->layout = s->aa ? LBM_LAYOUT_AA : LBM_LAYOUT_AB;
    o->force_1e4 = s->geom.storage == LBM_STORE_BF16 ? 0 : 1;
    return LBM_OK;
}

}  // extern "C"

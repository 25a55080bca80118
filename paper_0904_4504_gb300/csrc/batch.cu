// batch.cu -- many lattice instances of uneven sizes advanced by one persistent cooperative kernel
// (lbm_batch_* in include/lbm.h).
//
// Each instance is an ordinary simulation (lbm_create: geometry, buffers, force scratch and
// history) plus a device drive table of its own length.  A run of K steps is one cooperative
// launch of batch_kernel: its grid (every SM full) walks the tiles of all unfinished instances,
// round robin, and meets at a bounded grid barrier between steps.  The launch is a node of a CUDA
// graph that is built once per launch shape and replayed with new arguments.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "lbm.h"
#include "runtime.h"
#include "step_kernel.cuh"

using namespace lbm;

namespace {

struct Slot {
    lbm_sim* sim = nullptr;
    long long start = 0;      // batch step of the instance's step 0
    long long nsteps = 0;
    double* d_drive = nullptr;   // [nsteps] drive, then [nsteps] of it in FP32 (same allocation)
    size_t bytes = 0;
};

constexpr long long kDefaultBarrierLimit = 4000000000ll;  // clock cycles (about 2 s at 2 GHz)

}  // namespace

constexpr int kSubStreams = 16;

struct lbm_batch {
    int device = 0, Q = 0, storage = 0, collision = 0;
    int mode = LBM_BATCH_STREAMS;
    int variant = -1;                     // kernel of instances added in the streams mode (-1: default)
    cudaStream_t sub[kSubStreams] = {};   // instance launches (streams mode), one chain per instance
    cudaEvent_t ev_fork = nullptr, ev_join[kSubStreams] = {};
    int bx = 32, by = 4;
    size_t budget = 0, used = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<Slot> slots;
    long long gstep = 0;
    // device arrays of the launch
    BatchInst* d_insts = nullptr;
    size_t insts_cap = 0;
    int2* d_tiles = nullptr;
    size_t tiles_cap = 0;
    int ntiles = 0;
    unsigned int* d_bar = nullptr;  // [0] count, [1] generation
    int* d_err = nullptr;
    long long bar_limit = kDefaultBarrierLimit;
    bool dirty = true;
    BatchKernelFn kernel = nullptr;
    int max_blocks = 0;             // co-resident blocks of the whole GPU
    // graph of one cooperative launch, re-parameterized for every run
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    int graph_grid = 0;
    bool use_graph = true;
    // launch arguments (addresses stay valid for the graph's lifetime)
    const BatchInst* a_insts = nullptr;
    const int2* a_tiles = nullptr;
    int a_ntiles = 0;
    long long a_step0 = 0;
    int a_nsteps = 0;
    GridBarrier a_bar{};
    long long launches = 0;
    double lattice_updates = 0.0;   // fluid-node updates enqueued
};

namespace {

#define BCUDA(expr)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return set_error(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", \
                             #expr, cudaGetErrorString(e_));                                     \
    } while (0)

int check_batch(lbm_batch* b) {
    if (!b) return set_error(LBM_EINVAL, "null batch");
    BCUDA(cudaSetDevice(b->device));
    return LBM_OK;
}

bool slot_live(const Slot& s) { return s.sim != nullptr; }

bool slot_running(const lbm_batch* b, const Slot& s) {
    return s.sim && b->gstep - s.start < s.nsteps;
}

void free_graph(lbm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->node = nullptr;
    b->graph_grid = 0;
}

// Device bytes of one instance (populations, geometry arrays, force history, drive table).
size_t footprint(const HostLattice& H, int nx, int ny, int storage, int layout, long nsteps, int bx, int by) {
    const size_t es = storage_size(storage);
    const size_t align = 128 / es;
    const size_t pitch = (nx + align - 1) / align * align;
    const size_t plane = (size_t)ny * pitch;
    const size_t tiles = (size_t)((nx + bx - 1) / bx) * ((ny + by - 1) / by);
    const size_t hist = std::max<size_t>(1024, (size_t)nsteps);
    const size_t nbuf = layout == LBM_LAYOUT_AA ? 1 : 2;
    return nbuf * plane * H.Q * es + plane * (1 + sizeof(ulonglong2)) + tiles * (sizeof(int) + 2 * sizeof(double2)) +
           hist * sizeof(double2) + (size_t)nsteps * (sizeof(double) + sizeof(float)) + 4096;
}

// Rebuild the per-instance launch table and the tile list of the unfinished instances.
int rebuild(lbm_batch* b) {
    std::vector<BatchInst> insts(std::max<size_t>(1, b->slots.size()));
    std::vector<int2> tiles;
    for (size_t k = 0; k < b->slots.size(); ++k) {
        const Slot& s = b->slots[k];
        BatchInst& I = insts[k];
        std::memset((void*)&I, 0, sizeof(I));
        I.nsteps = 0;
        if (!slot_live(s)) continue;
        const SimView v = sim_view(s.sim);
        I.base = v.inst;
        I.buf[0] = v.buf[0];
        I.buf[1] = v.buf[1];
        I.drive = s.d_drive;
        I.drive_f = reinterpret_cast<const float*>(s.d_drive + s.nsteps);
        I.history = v.history;
        I.start = s.start;
        I.nsteps = s.nsteps;
        if (!slot_running(b, s)) continue;
        for (int t = 0; t < v.inst.ntiles; ++t) tiles.push_back(make_int2((int)k, t));
    }
    if (insts.size() > b->insts_cap) {
        cudaFree(b->d_insts);
        b->d_insts = nullptr;
        BCUDA(cudaMalloc((void**)&b->d_insts, insts.size() * sizeof(BatchInst)));
        b->insts_cap = insts.size();
    }
    if (tiles.size() > b->tiles_cap || !b->d_tiles) {
        cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        const size_t cap = std::max<size_t>(tiles.size(), 1);
        BCUDA(cudaMalloc((void**)&b->d_tiles, cap * sizeof(int2)));
        b->tiles_cap = cap;
    }
    BCUDA(cudaMemcpyAsync(b->d_insts, insts.data(), insts.size() * sizeof(BatchInst), cudaMemcpyHostToDevice,
                          b->stream));
    if (!tiles.empty())
        BCUDA(cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice,
                              b->stream));
    // the host vectors die here: wait for the copies
    BCUDA(cudaStreamSynchronize(b->stream));
    b->ntiles = (int)tiles.size();
    b->dirty = false;
    return LBM_OK;
}

int launch(lbm_batch* b, int grid, long long step0, int nsteps) {
    b->a_insts = b->d_insts;
    b->a_tiles = b->d_tiles;
    b->a_ntiles = b->ntiles;
    b->a_step0 = step0;
    b->a_nsteps = nsteps;
    b->a_bar = GridBarrier{b->d_bar, b->d_bar + 1, b->d_err, b->bar_limit};
    void* args[] = {(void*)&b->a_insts, (void*)&b->a_tiles, (void*)&b->a_ntiles, (void*)&b->a_step0,
                    (void*)&b->a_nsteps, (void*)&b->a_bar};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(b->kernel);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(b->bx, b->by);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    if (b->use_graph) {
        cudaError_t e = cudaSuccess;
        if (!b->exec || b->graph_grid != grid) {
            free_graph(b);
            e = cudaGraphCreate(&b->graph, 0);
            if (e == cudaSuccess) e = cudaGraphAddKernelNode(&b->node, b->graph, nullptr, 0, &kp);
            if (e == cudaSuccess) {
                cudaLaunchAttributeValue v{};
                v.cooperative = 1;
                e = cudaGraphKernelNodeSetAttribute(b->node, cudaLaunchAttributeCooperative, &v);
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e == cudaSuccess) b->graph_grid = grid;
        } else {
            e = cudaGraphExecKernelNodeSetParams(b->exec, b->node, &kp);
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
        if (e == cudaSuccess) return LBM_OK;
        // graphs with cooperative nodes unavailable: launch directly from now on
        cudaGetLastError();
        free_graph(b);
        b->use_graph = false;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(b->bx, b->by);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BCUDA(cudaLaunchKernelExC(&cfg, b->kernel, args));
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(int lattice, int storage, int collision, size_t device_budget_bytes, lbm_batch** out) {
    clear_error();
    if (!out) return set_error(LBM_EINVAL, "null output handle");
    *out = nullptr;
    HostLattice H;
    if (!host_lattice(lattice, H)) return set_error(LBM_EINVAL, "lattice must be LBM_D2Q9 or LBM_D2Q37");
    if (!storage_size(storage)) return set_error(LBM_EINVAL, "bad storage type %d", storage);
    if (collision != LBM_COLL_BGK && collision != LBM_COLL_REGULARIZED) return set_error(LBM_EINVAL, "bad collision");
    BatchKernelFn k = find_batch_kernel(lattice, storage, collision);
    if (!k) return set_error(LBM_EINVAL, "no batch kernel for this lattice/storage/collision");
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return set_error(LBM_ENOMEM, "host allocation");
    b->Q = lattice;
    b->storage = storage;
    b->collision = collision;
    b->kernel = k;
    int rc = LBM_OK;
    auto fail = [&](int code) {
        lbm_batch_destroy(b);
        return code;
    };
    if (cudaGetDevice(&b->device) != cudaSuccess) return fail(set_error(LBM_ECUDA, "no CUDA device"));
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(set_error(LBM_ECUDA, "cudaMemGetInfo"));
    const size_t margin = (size_t)1 << 30;
    b->budget = device_budget_bytes ? device_budget_bytes : (free_b > margin ? free_b - margin : free_b / 2);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(set_error(LBM_ECUDA, "stream creation"));
    b->own_stream = true;
    if (cudaMalloc((void**)&b->d_bar, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess)
        return fail(set_error(LBM_ENOMEM, "batch barrier"));
    for (int k = 0; k < kSubStreams; ++k)
        if (cudaStreamCreateWithFlags(&b->sub[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess)
            return fail(set_error(LBM_ECUDA, "stream creation"));
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(set_error(LBM_ECUDA, "event creation"));
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b->kernel, b->bx * b->by, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || per_sm < 1)
        return fail(set_error(LBM_ECUDA, "occupancy query of the batch kernel"));
    b->max_blocks = per_sm * sms;
    (void)rc;
    *out = b;
    return LBM_OK;
}

int lbm_batch_footprint(const lbm_instance_desc* d, size_t* bytes) {
    if (!d || !bytes) return set_error(LBM_EINVAL, "null argument");
    HostLattice H;
    if (!host_lattice(d->lattice, H)) return set_error(LBM_EINVAL, "unknown lattice %d", d->lattice);
    if (!storage_size(d->geom.storage)) return set_error(LBM_EINVAL, "bad storage type");
    if (d->nx < 1 || d->ny < 1 || d->nsteps < 0) return set_error(LBM_EINVAL, "bad size");
    *bytes = footprint(H, d->nx, d->ny, d->geom.storage, d->geom.layout, d->nsteps, 32, 4);
    return LBM_OK;
}

int lbm_batch_add(lbm_batch* b, const lbm_instance_desc* d, int* slot) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (!d || !slot) return set_error(LBM_EINVAL, "null argument");
    if (d->lattice != b->Q || d->geom.storage != b->storage || d->geom.collision != b->collision)
        return set_error(LBM_EINVAL, "instance lattice/storage/collision differ from the batch's");
    if (d->nsteps < 1) return set_error(LBM_EINVAL, "nsteps must be >= 1");
    if (b->mode == LBM_BATCH_PERSISTENT && d->geom.wall_scheme != LBM_SCHEME_BOUNCEBACK)
        return set_error(LBM_EINVAL, "the persistent batch kernel is built for bounce-back walls only");
    if (b->mode == LBM_BATCH_PERSISTENT && d->geom.layout != LBM_LAYOUT_AB)
        return set_error(LBM_EINVAL, "the persistent batch kernel runs the two-buffer layout only");
    HostLattice H;
    host_lattice(d->lattice, H);
    const size_t bytes = footprint(H, d->nx, d->ny, d->geom.storage, d->geom.layout, d->nsteps, b->bx, b->by);
    if (b->used + bytes > b->budget)
        return set_error(LBM_ENOMEM, "instance needs %zu bytes, %zu of the %zu-byte budget are free", bytes,
                         b->budget - b->used, b->budget);
    lbm_sim* sim = nullptr;
    rc = lbm_create(d->lattice, d->nx, d->ny, d->tau, d->omega, &d->geom, &sim);
    if (rc) return rc;
    auto undo = [&](int code) {
        lbm_destroy(sim);
        return code;
    };
    int id = -1;
    for (size_t k = 0; k < b->slots.size(); ++k)
        if (!slot_live(b->slots[k])) { id = (int)k; break; }
    if (id < 0) id = (int)b->slots.size();
    // kernel shape, history and stream, on the instance's own stream first, so that adding an
    // instance does not wait for a run of the batch that may be in flight
    if (b->mode == LBM_BATCH_PERSISTENT) sim_disable_stream_offset(sim);  // the kernel reads fixed params
    // default kernels, fastest measured in this mode: for D2Q37, the staged kernel with three rows
    // per thread (27) for 16-bit storage and the plain kernel with 7 resident blocks per SM (2) for
    // FP32; 16-bit D2Q9 takes the staged kernel 10; else the plain kernel
    const bool half = b->storage == LBM_STORE_BF16 || b->storage == LBM_STORE_F16;
    const int want = b->variant >= 0 ? b->variant
                     : half ? (b->Q == 37 ? 27 : 10)
                     : (b->Q == 37 && b->storage == LBM_STORE_F32) ? 2 : 0;
    if (b->mode == LBM_BATCH_PERSISTENT || want == 0 || lbm_set_variant(sim, want) != LBM_OK)
        rc = lbm_set_tile(sim, b->bx, b->by);
    if (rc) return undo(rc);
    clear_error();
    // (+1: an in-place even step also writes the force of the step after it)
    if ((rc = sim_reserve(sim, (size_t)d->nsteps + 1))) return undo(rc);
    if ((rc = lbm_set_stream(sim, b->mode == LBM_BATCH_STREAMS ? b->sub[id % kSubStreams] : b->stream)))
        return undo(rc);
    // drive table: nsteps doubles followed by the same values as nsteps floats
    const size_t N = (size_t)d->nsteps;
    std::vector<double> table(N + (N + 1) / 2, 0.0);
    float* tf = reinterpret_cast<float*>(table.data() + N);
    for (size_t n = 0; n < N; ++n) {
        table[n] = drive_value(d->geom.drive, d->geom.u0, d->omega, (long)n);
        tf[n] = (float)table[n];
    }
    double* drv = nullptr;
    if (cudaMalloc((void**)&drv, table.size() * sizeof(double)) != cudaSuccess)
        return undo(set_error(LBM_ENOMEM, "drive table"));
    if (cudaMemcpy(drv, table.data(), table.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(drv);
        return undo(set_error(LBM_ECUDA, "drive table upload"));
    }
    Slot s;
    s.sim = sim;
    s.start = b->gstep;
    s.nsteps = d->nsteps;
    s.d_drive = drv;
    s.bytes = bytes;
    if (id == (int)b->slots.size()) b->slots.push_back(s);
    else b->slots[id] = s;
    b->used += bytes;
    b->dirty = true;
    *slot = id;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch* b, long steps) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (steps < 0) return set_error(LBM_EINVAL, "negative step count");
    if (steps == 0) return LBM_OK;
    if (steps > (1l << 30)) return set_error(LBM_EINVAL, "too many steps in one run");
    // drop instances that finished before this run
    for (const Slot& s : b->slots)
        if (slot_live(s) && !slot_running(b, s) && b->ntiles > 0) b->dirty = true;
    if (b->mode == LBM_BATCH_STREAMS) {
        // every running instance advances on its own stream chain; the sub-streams follow the
        // batch stream's earlier work and the batch stream waits for theirs at the end
        BCUDA(cudaEventRecord(b->ev_fork, b->stream));
        for (int k = 0; k < kSubStreams; ++k) BCUDA(cudaStreamWaitEvent(b->sub[k], b->ev_fork, 0));
        for (long k = 0; k < steps; ++k) {
            for (Slot& s : b->slots) {
                if (!slot_live(s)) continue;
                const long long n = b->gstep + k - s.start;
                if (n < 0 || n >= s.nsteps) continue;
                if ((rc = lbm_step(s.sim, 1))) return rc;
                b->lattice_updates += (double)sim_view(s.sim).n_fluid;
                ++b->launches;
            }
        }
        for (int k = 0; k < kSubStreams; ++k) {
            BCUDA(cudaEventRecord(b->ev_join[k], b->sub[k]));
            BCUDA(cudaStreamWaitEvent(b->stream, b->ev_join[k], 0));
        }
        b->gstep += steps;
        return LBM_OK;
    }
    if (b->dirty && (rc = rebuild(b))) return rc;
    bool any = false;
    for (const Slot& s : b->slots) any = any || slot_running(b, s);
    if (any && b->ntiles > 0) {
        const int grid = std::min(b->ntiles, b->max_blocks);
        BCUDA(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned int), b->stream));
        if ((rc = launch(b, grid, b->gstep, (int)steps))) return rc;
        ++b->launches;
    }
    for (Slot& s : b->slots) {
        if (!slot_live(s)) continue;
        const long long before = std::max<long long>(0, std::min(s.nsteps, b->gstep - s.start));
        const long long after = std::max<long long>(0, std::min(s.nsteps, b->gstep + steps - s.start));
        if (after > before) {
            sim_advance(s.sim, (long)(after - before));
            b->lattice_updates += (double)(after - before) * (double)sim_view(s.sim).n_fluid;
        }
    }
    b->gstep += steps;
    return LBM_OK;
}

int lbm_batch_synchronize(lbm_batch* b) {
    int rc = check_batch(b);
    if (rc) return rc;
    BCUDA(cudaStreamSynchronize(b->stream));
    for (int k = 0; k < kSubStreams; ++k) BCUDA(cudaStreamSynchronize(b->sub[k]));
    for (const Slot& s : b->slots)
        if (slot_live(s) && (rc = lbm_synchronize(s.sim)) != LBM_OK) return rc;
    int err = 0;
    BCUDA(cudaMemcpy(&err, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & 2) return set_error(LBM_ETIMEOUT, "a grid-barrier wait of the batch kernel timed out; states are undefined");
    return LBM_OK;
}

int lbm_batch_status(lbm_batch* b, int slot, long* steps_done, long* nsteps) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (slot < 0 || slot >= (int)b->slots.size() || !slot_live(b->slots[slot]))
        return set_error(LBM_ERANGE, "no instance in slot %d", slot);
    const Slot& s = b->slots[slot];
    if (steps_done) *steps_done = (long)std::max<long long>(0, std::min(s.nsteps, b->gstep - s.start));
    if (nsteps) *nsteps = (long)s.nsteps;
    return LBM_OK;
}

lbm_sim* lbm_batch_instance(lbm_batch* b, int slot) {
    if (!b || slot < 0 || slot >= (int)b->slots.size()) return nullptr;
    return b->slots[slot].sim;
}

int lbm_batch_remove(lbm_batch* b, int slot) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (slot < 0 || slot >= (int)b->slots.size() || !slot_live(b->slots[slot]))
        return set_error(LBM_ERANGE, "no instance in slot %d", slot);
    BCUDA(cudaStreamSynchronize(b->stream));
    for (int k = 0; k < kSubStreams; ++k) BCUDA(cudaStreamSynchronize(b->sub[k]));
    Slot& s = b->slots[slot];
    lbm_destroy(s.sim);
    cudaFree(s.d_drive);
    b->used -= s.bytes;
    s = Slot();
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_set_barrier_limit(lbm_batch* b, long long cycles) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (cycles < 0) return set_error(LBM_EINVAL, "negative limit");
    b->bar_limit = cycles;
    return LBM_OK;
}

int lbm_batch_info(lbm_batch* b, lbm_batch_info_t* o) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (!o) return set_error(LBM_EINVAL, "null output");
    o->lattice = b->Q;
    o->storage = b->storage;
    o->collision = b->collision;
    o->live = o->running = 0;
    o->fluid_running = 0;
    o->bytes_per_step = 0;
    for (const Slot& s : b->slots) {
        if (!slot_live(s)) continue;
        ++o->live;
        if (slot_running(b, s)) {
            const SimView v = sim_view(s.sim);
            ++o->running;
            o->fluid_running += v.n_fluid;
            o->bytes_per_step += 2 * (size_t)v.Q * v.esize * v.n_fluid;
        }
    }
    o->batch_steps = b->gstep;
    o->launches = b->launches;
    o->lattice_updates = b->lattice_updates;
    o->budget_bytes = b->budget;
    o->used_bytes = b->used;
    o->max_blocks = b->max_blocks;
    o->uses_graph = (b->mode == LBM_BATCH_PERSISTENT && b->use_graph) ? 1 : 0;
    o->mode = b->mode;
    o->block_x = b->bx;
    o->block_y = b->by;
    return LBM_OK;
}

int lbm_batch_set_stream(lbm_batch* b, void* stream) {
    int rc = check_batch(b);
    if (rc) return rc;
    BCUDA(cudaStreamSynchronize(b->stream));
    if (b->own_stream) cudaStreamDestroy(b->stream);
    b->stream = (cudaStream_t)stream;
    b->own_stream = false;
    if (b->mode == LBM_BATCH_PERSISTENT)
        for (Slot& s : b->slots)
            if (slot_live(s) && (rc = lbm_set_stream(s.sim, stream))) return rc;
    return LBM_OK;
}

int lbm_batch_set_mode(lbm_batch* b, int mode) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (mode != LBM_BATCH_PERSISTENT && mode != LBM_BATCH_STREAMS) return set_error(LBM_EINVAL, "bad batch mode");
    for (const Slot& s : b->slots)
        if (slot_live(s)) return set_error(LBM_EINVAL, "set the mode before adding instances");
    b->mode = mode;
    return LBM_OK;
}

int lbm_batch_set_variant(lbm_batch* b, int variant) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (variant < -1) return set_error(LBM_EINVAL, "bad variant %d", variant);
    b->variant = variant;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (Slot& s : b->slots) {
        if (s.sim) lbm_destroy(s.sim);
        cudaFree(s.d_drive);
    }
    for (int k = 0; k < kSubStreams; ++k) {
        if (b->sub[k]) {
            cudaStreamSynchronize(b->sub[k]);
            cudaStreamDestroy(b->sub[k]);
        }
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    free_graph(b);
    cudaFree(b->d_insts);
    cudaFree(b->d_tiles);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

// batch.cu -- many lattice instances of uneven sizes advanced together (lbm_batch_* in include/lbm.h).
//
// Each instance is an ordinary simulation (lbm_create: geometry, buffers, force scratch and
// history).  Two modes run them:
//  * persistent: a run of K steps is one launch of the persistent kernel (pbatch.cuh), whose blocks
//    take (step, tile) items of every running instance from a queue and wait only for the tiles
//    within reach of theirs; each instance adds a table of its per-step constants, per-tile step
//    counters and a ring of force slots.  The launch (queue reset + kernel) is a CUDA graph built
//    once per grid size and replayed with new arguments.
//  * streams: every instance's step is a launch of the single-instance kernel on one of 16
//    parallel streams.
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
    // persistent mode: one allocation holding the per-step constants [nsteps], the band counters
    // [<= nty], the force ring [kRing][nslots], its tickets [kRing] and finish marks [kRing]
    unsigned char* d_pb = nullptr;
    size_t off_done = 0, off_ring = 0, off_tickets = 0, off_fin = 0;
    size_t bytes = 0;
};

constexpr long long kDefaultWaitLimit = 4000000000ll;  // clock cycles (about 2 s at 2 GHz)

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
    PInst* d_insts = nullptr;
    size_t insts_cap = 0;
    int4* d_segs = nullptr;         // (instance, band, tile column, 0) of the running instances
    size_t segs_cap = 0;
    int nsegs = 0;
    int seg_tiles = 8;              // tile rows per work item (strip) of the persistent kernel
    int pinned_seg = 0;             // strip length fixed by the seg_tiles in use at the first run
    unsigned long long* d_queue = nullptr;  // work-item counter of the persistent kernel
    int* d_err = nullptr;
    long long wait_limit = kDefaultWaitLimit;
    bool dirty = true;
    int pvariant = -1;              // persistent kernel: the variant whose tile code it runs (-1: not chosen)
    PbKernel kernel{};
    int max_blocks = 0;             // co-resident blocks of the whole GPU
    // graph of one launch (queue reset, kernel), re-parameterized for every run
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    int graph_grid = 0;
    bool use_graph = true;
    PbArgs a_args{};                // launch arguments (the address stays valid for the graph's lifetime)
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

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Layout of a persistent-mode instance's allocation (see Slot); returns its size.
size_t pb_layout(long long nsteps, int nty, int nslots, Slot* s) {
    size_t off = align_up((size_t)nsteps * sizeof(StepConst), 256);
    const size_t done = off;
    off = align_up(off + (size_t)nty * sizeof(int), 256);
    const size_t ring = off;
    off = align_up(off + (size_t)kRing * (size_t)std::max(1, nslots) * sizeof(double2), 256);
    const size_t tickets = off;
    off = align_up(off + kRing * sizeof(unsigned int), 256);
    const size_t fin = off;
    off = align_up(off + kRing * sizeof(int), 256);
    if (s) {
        s->off_done = done;
        s->off_ring = ring;
        s->off_tickets = tickets;
        s->off_fin = fin;
    }
    return off;
}

// Device bytes of one instance (populations, geometry arrays, force history, and in the persistent
// mode its step table, tile counters and force ring; the tile shape bx x by).
size_t footprint(const HostLattice& H, int nx, int ny, int storage, int layout, long nsteps, int bx, int by) {
    const size_t es = storage_size(storage);
    const size_t align = 128 / es;
    const size_t pitch = (nx + align - 1) / align * align;
    const size_t plane = (size_t)ny * pitch;
    const size_t tiles = (size_t)((nx + bx - 1) / bx) * ((ny + by - 1) / by);
    const size_t hist = std::max<size_t>(1024, (size_t)nsteps + 1);
    const size_t nbuf = layout == LBM_LAYOUT_AA ? 1 : 2;
    return nbuf * plane * H.Q * es + plane * (1 + sizeof(ulonglong2)) + tiles * (sizeof(int) + 2 * sizeof(double2)) +
           hist * sizeof(double2) + pb_layout(nsteps, (int)tiles, (int)tiles, nullptr) + 4096;
}

// Rebuild the per-instance launch table and the strip list of the unfinished instances.
int rebuild(lbm_batch* b) {
    std::vector<PInst> insts(std::max<size_t>(1, b->slots.size()));
    std::vector<int4> segs;
    for (size_t k = 0; k < b->slots.size(); ++k) {
        const Slot& s = b->slots[k];
        PInst& I = insts[k];
        std::memset((void*)&I, 0, sizeof(I));
        if (!slot_live(s)) continue;
        const SimView v = sim_view(s.sim);
        if (v.maps) std::memcpy((void*)I.maps, (const void*)v.maps, sizeof(I.maps));
        I.base = v.inst;
        I.buf[0] = v.buf[0];
        I.buf[1] = v.buf[1];
        I.steps = reinterpret_cast<const StepConst*>(s.d_pb);
        I.history = v.history;
        I.done = reinterpret_cast<int*>(s.d_pb + s.off_done);
        I.ring = reinterpret_cast<double2*>(s.d_pb + s.off_ring);
        I.tickets = reinterpret_cast<unsigned int*>(s.d_pb + s.off_tickets);
        I.fin = reinterpret_cast<int*>(s.d_pb + s.off_fin);
        I.start = s.start;
        I.nsteps = s.nsteps;
        I.bx = v.bx;
        I.by = v.by;
        I.nty = (v.ny + v.by - 1) / v.by;
        const int ntx = v.inst.ntx, S = b->seg_tiles;
        I.band = S;
        I.nseg = ntx;
        if (!slot_running(b, s)) continue;
        // the columns of a band follow each other, so that they run side by side
        for (int band = 0; band * S < I.nty; ++band)
            for (int tx = 0; tx < ntx; ++tx) segs.push_back(make_int4((int)k, band, tx, 0));
    }
    if (insts.size() > b->insts_cap) {
        cudaFree(b->d_insts);
        b->d_insts = nullptr;
        BCUDA(cudaMalloc((void**)&b->d_insts, insts.size() * sizeof(PInst)));
        b->insts_cap = insts.size();
    }
    if (segs.size() > b->segs_cap || !b->d_segs) {
        cudaFree(b->d_segs);
        b->d_segs = nullptr;
        const size_t cap = std::max<size_t>(segs.size(), 1);
        BCUDA(cudaMalloc((void**)&b->d_segs, cap * sizeof(int4)));
        b->segs_cap = cap;
    }
    BCUDA(cudaMemcpyAsync(b->d_insts, insts.data(), insts.size() * sizeof(PInst), cudaMemcpyHostToDevice,
                          b->stream));
    if (!segs.empty())
        BCUDA(cudaMemcpyAsync(b->d_segs, segs.data(), segs.size() * sizeof(int4), cudaMemcpyHostToDevice,
                              b->stream));
    // the host vectors die here: wait for the copies
    BCUDA(cudaStreamSynchronize(b->stream));
    b->nsegs = (int)segs.size();
    b->pinned_seg = b->seg_tiles;
    b->dirty = false;
    return LBM_OK;
}

// One run of the persistent kernel: a graph of two nodes, the reset of the work-item counter and
// the kernel, built once per grid size; later runs only update the kernel's arguments.
int launch(lbm_batch* b, int grid, long long step0, int nsteps) {
    b->a_args = PbArgs{b->d_insts, b->d_segs, b->nsegs, nsteps, step0, b->d_queue, 0ull, b->d_err, b->wait_limit};
    void* args[] = {(void*)&b->a_args};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(b->kernel.func);
    kp.gridDim = dim3(grid);
    kp.blockDim = b->kernel.block;
    kp.sharedMemBytes = (unsigned)b->kernel.smem;
    kp.kernelParams = args;
    kp.extra = nullptr;
    if (b->use_graph) {
        cudaError_t e = cudaSuccess;
        if (!b->exec || b->graph_grid != grid) {
            free_graph(b);
            cudaGraphNode_t reset = nullptr;
            cudaMemsetParams mp{};
            mp.dst = b->d_queue;
            mp.value = 0;
            mp.elementSize = 4;
            mp.width = 2;   // the 64-bit counter as two 32-bit words
            mp.height = 1;
            mp.pitch = 0;
            e = cudaGraphCreate(&b->graph, 0);
            if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&reset, b->graph, nullptr, 0, &mp);
            if (e == cudaSuccess) e = cudaGraphAddKernelNode(&b->node, b->graph, &reset, 1, &kp);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (e == cudaSuccess) b->graph_grid = grid;
        } else {
            e = cudaGraphExecKernelNodeSetParams(b->exec, b->node, &kp);
        }
        if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
        if (e == cudaSuccess) return LBM_OK;
        // graphs unavailable: launch directly from now on
        cudaGetLastError();
        free_graph(b);
        b->use_graph = false;
    }
    BCUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), b->stream));
    BCUDA(cudaLaunchKernel(b->kernel.func, dim3(grid), b->kernel.block, args, (size_t)b->kernel.smem, b->stream));
    return LBM_OK;
}

// The persistent kernel's default variant for the batch's class: staged 64 x 3 tiles (27) with
// 16-bit storage, plain 32 x 4 tiles otherwise (2 for D2Q37 FP32, else 0).
int default_pvariant(const lbm_batch* b) {
    if (b->storage == LBM_STORE_BF16 || b->storage == LBM_STORE_F16) return 27;
    return (b->Q == 37 && b->storage != LBM_STORE_F64) ? 2 : 0;
}

// Choose the persistent kernel of the batch's class by variant (-1: the default).
int choose_kernel(lbm_batch* b, int variant) {
    if (variant < 0) variant = default_pvariant(b);
    const PbKernel k = find_pbatch_kernel(b->Q, b->storage, b->collision, variant);
    if (!k.func)
        return set_error(LBM_EINVAL, "the persistent kernel runs no variant %d for this lattice/storage/collision",
                         variant);
    if (k.smem > 0)
        BCUDA(cudaFuncSetAttribute(k.func, cudaFuncAttributeMaxDynamicSharedMemorySize, k.smem));
    int per_sm = 0, sms = 0;
    BCUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.func, (int)(k.block.x * k.block.y), k.smem));
    BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    if (per_sm < 1) return set_error(LBM_ECUDA, "the persistent kernel does not fit on an SM");
    b->kernel = k;
    b->pvariant = variant;
    b->bx = k.tile_x;
    b->by = k.tile_y;
    b->max_blocks = per_sm * sms;
    free_graph(b);
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
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return set_error(LBM_ENOMEM, "host allocation");
    b->Q = lattice;
    b->storage = storage;
    b->collision = collision;
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
    if (cudaMalloc((void**)&b->d_queue, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&b->d_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(b->d_queue, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(b->d_err, 0, sizeof(int)) != cudaSuccess)
        return fail(set_error(LBM_ENOMEM, "batch work counter"));
    for (int k = 0; k < kSubStreams; ++k)
        if (cudaStreamCreateWithFlags(&b->sub[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess)
            return fail(set_error(LBM_ECUDA, "stream creation"));
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(set_error(LBM_ECUDA, "event creation"));
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
    if (b->mode == LBM_BATCH_PERSISTENT && !b->kernel.func && (rc = choose_kernel(b, -1))) return rc;
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
    const bool half = b->storage == LBM_STORE_BF16 || b->storage == LBM_STORE_F16;
    if (b->mode == LBM_BATCH_PERSISTENT) {
        // the instance's tile shape is the persistent kernel's: that of the variant whose tile code
        // it runs (for staged tiles also the load boxes)
        rc = b->pvariant ? lbm_set_variant(sim, b->pvariant) : lbm_set_tile(sim, 32, 4);
    } else {
        // default kernels, fastest measured in this mode: for D2Q37, the staged kernel with three
        // rows per thread (27) for 16-bit storage and the plain kernel with 7 resident blocks per SM
        // (2) for FP32; 16-bit D2Q9 takes the four-nodes-per-thread kernel (30); else the plain
        // kernel
        const int want = b->variant >= 0 ? b->variant
                         : half ? (b->Q == 37 ? 27 : 30)
                         : (b->Q == 37 && b->storage == LBM_STORE_F32) ? 2 : 0;
        if (want == 0 || lbm_set_variant(sim, want) != LBM_OK) rc = lbm_set_tile(sim, b->bx, b->by);
    }
    if (rc) return undo(rc);
    clear_error();
    // (+1: an in-place even step also writes the force of the step after it)
    if ((rc = sim_reserve(sim, (size_t)d->nsteps + 1))) return undo(rc);
    if ((rc = lbm_set_stream(sim, b->mode == LBM_BATCH_STREAMS ? b->sub[id % kSubStreams] : b->stream)))
        return undo(rc);
    Slot s;
    if (b->mode == LBM_BATCH_PERSISTENT) {
        // per-step constants, tile counters (0: no step done) and the force ring (entry j free,
        // as if the step j - kRing had left it)
        const SimView v = sim_view(sim);
        const size_t pb = pb_layout(d->nsteps, (v.ny + v.by - 1) / v.by, v.nslots, &s);
        std::vector<unsigned char> host(pb, 0);
        sim_step_constants(sim, d->nsteps, reinterpret_cast<StepConst*>(host.data()));
        int* fin = reinterpret_cast<int*>(host.data() + s.off_fin);
        for (int j = 0; j < kRing; ++j) fin[j] = j - kRing + 1;
        if (cudaMalloc((void**)&s.d_pb, pb) != cudaSuccess) return undo(set_error(LBM_ENOMEM, "batch step table"));
        if (cudaMemcpy(s.d_pb, host.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(s.d_pb);
            return undo(set_error(LBM_ECUDA, "batch step table upload"));
        }
    }
    s.sim = sim;
    s.start = b->gstep;
    s.nsteps = d->nsteps;
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
        if (slot_live(s) && !slot_running(b, s) && b->nsegs > 0) b->dirty = true;
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
    if (any && b->nsegs > 0) {
        const long long items = (long long)b->nsegs * steps;
        const int grid = (int)std::min<long long>(items, b->max_blocks);
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
    if (err & 8)
        return set_error(LBM_ETIMEOUT, "a bounded wait of the persistent batch kernel ran out; states are undefined");
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
    cudaFree(s.d_pb);
    b->used -= s.bytes;
    s = Slot();
    b->dirty = true;
    return LBM_OK;
}

int lbm_batch_set_barrier_limit(lbm_batch* b, long long cycles) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (cycles < 0) return set_error(LBM_EINVAL, "negative limit");
    b->wait_limit = cycles;
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
    if (mode == LBM_BATCH_PERSISTENT) {
        // the persistent kernel of the variant set before, if it runs one; the class's default otherwise
        const int v = (b->variant >= 0 && find_pbatch_kernel(b->Q, b->storage, b->collision, b->variant).func)
                          ? b->variant : -1;
        if ((rc = choose_kernel(b, v))) return rc;
    } else {
        b->bx = 32;
        b->by = 4;
    }
    b->mode = mode;
    return LBM_OK;
}

int lbm_batch_set_segment(lbm_batch* b, int tiles) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (tiles < 1 || tiles > 1024) return set_error(LBM_EINVAL, "strip of %d tile rows: need 1..1024", tiles);
    // the band counters count strips, so the length is fixed once the persistent kernel has run
    if (b->pinned_seg && tiles != b->pinned_seg)
        return set_error(LBM_EINVAL, "the strip length is fixed after the first persistent run");
    b->seg_tiles = tiles;
    return LBM_OK;
}

int lbm_batch_set_variant(lbm_batch* b, int variant) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (variant < -1) return set_error(LBM_EINVAL, "bad variant %d", variant);
    if (b->mode == LBM_BATCH_PERSISTENT) {
        for (const Slot& s : b->slots)
            if (slot_live(s)) return set_error(LBM_EINVAL, "set the persistent kernel before adding instances");
        if ((rc = choose_kernel(b, variant))) return rc;
    }
    b->variant = variant;
    return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, const lbm_instance_desc* descs, int n, int steps, lbm_batch_tune_entry* out, int cap,
                   int* n_out) {
    int rc = check_batch(b);
    if (rc) return rc;
    if (!descs || n < 1 || steps < 1 || !n_out || (cap > 0 && !out))
        return set_error(LBM_EINVAL, "need instance descriptions, steps >= 1 and an output");
    // candidates: streams mode, the step kernels of the class; persistent mode, its tile paths
    // (staged 27 and 28, plain 2 and 0) times the strip lengths
    std::vector<lbm_batch_tune_entry> cand;
    if (b->mode == LBM_BATCH_STREAMS) {
        for (int v : {0, 1, 2, 10, 20, 26, 27, 28, 30}) cand.push_back(lbm_batch_tune_entry{v, 0, 0.0});
    } else {
        for (int v : {27, 28, 2, 0})
            if (find_pbatch_kernel(b->Q, b->storage, b->collision, v).func)
                for (int sg : {4, 8, 12}) cand.push_back(lbm_batch_tune_entry{v, sg, 0.0});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return set_error(LBM_ECUDA, "event creation");
    }
    int k = 0;
    const int warm = 2;
    for (auto& e : cand) {
        lbm_batch* t = nullptr;
        if ((rc = lbm_batch_create(b->Q, b->storage, b->collision, b->budget, &t))) break;
        rc = lbm_batch_set_mode(t, b->mode);
        if (rc == LBM_OK) rc = lbm_batch_set_variant(t, e.variant);
        if (rc == LBM_OK && b->mode == LBM_BATCH_PERSISTENT) rc = lbm_batch_set_segment(t, e.segment);
        bool usable = rc == LBM_OK;
        int added = 0;
        for (int j = 0; usable && j < n; ++j) {
            lbm_instance_desc d = descs[j];
            d.nsteps = warm + steps;
            int slot = -1;
            const int r = lbm_batch_add(t, &d, &slot);
            if (r == LBM_ENOMEM) break;  // the clones fill the budget: time the ones that fit
            if (r != LBM_OK) { rc = r; usable = false; break; }
            // a streams-mode variant that the class does not build falls back to the plain kernel:
            // not a distinct candidate
            if (b->mode == LBM_BATCH_STREAMS && sim_view(t->slots[slot].sim).variant != e.variant) usable = false;
            ++added;
        }
        clear_error();
        if (usable && added > 0) {
            rc = lbm_batch_run(t, warm);
            if (rc == LBM_OK && cudaEventRecord(e0, t->stream) != cudaSuccess) rc = set_error(LBM_ECUDA, "event");
            if (rc == LBM_OK) rc = lbm_batch_run(t, steps);
            if (rc == LBM_OK && cudaEventRecord(e1, t->stream) != cudaSuccess) rc = set_error(LBM_ECUDA, "event");
            if (rc == LBM_OK) rc = lbm_batch_synchronize(t);
            if (rc == LBM_OK) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                e.us_per_step = 1000.0 * ms / steps;
                if (k < cap) out[k] = e;
                ++k;
            }
        } else if (rc == LBM_EINVAL) {
            rc = LBM_OK;  // candidate not built for this class
            clear_error();
        }
        lbm_batch_destroy(t);
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *n_out = k;
    return rc;
}

int lbm_batch_autotune(lbm_batch* b, const lbm_instance_desc* descs, int n, int steps, lbm_batch_tune_entry* best) {
    int rc = check_batch(b);
    if (rc) return rc;
    for (const Slot& s : b->slots)
        if (slot_live(s)) return set_error(LBM_EINVAL, "tune the batch before adding instances");
    lbm_batch_tune_entry e[32];
    int m = 0;
    if ((rc = lbm_batch_tune(b, descs, n, steps, e, 32, &m))) return rc;
    if (m == 0) return set_error(LBM_EINVAL, "no candidate could be timed");
    int k = 0;
    for (int j = 1; j < m; ++j)
        if (e[j].us_per_step < e[k].us_per_step) k = j;
    if ((rc = lbm_batch_set_variant(b, e[k].variant))) return rc;
    if (b->mode == LBM_BATCH_PERSISTENT && (rc = lbm_batch_set_segment(b, e[k].segment))) return rc;
    if (best) *best = e[k];
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (Slot& s : b->slots) {
        if (s.sim) lbm_destroy(s.sim);
        cudaFree(s.d_pb);
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
    cudaFree(b->d_segs);
    cudaFree(b->d_queue);
    cudaFree(b->d_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

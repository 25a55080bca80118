// runtime.h -- host-side helpers shared by the C-ABI translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "lbm.h"
#include "pbatch.cuh"

namespace lbm {

struct HostLattice {
    int Q = 0, R = 0;
    double theta = 0;
    int c[37][2] = {};
    double w[37] = {};
    int opp[37] = {};
};

bool host_lattice(int Q, HostLattice& H);
size_t storage_size(int storage);
int set_error(int code, const char* fmt, ...);
void clear_error();
const char* last_error();
int build_labels(int Q, int nx, int ny, const lbm_geometry& g, std::vector<uint8_t>& lab);
// A fluid node with blocked links: its offset in the unpadded grid (y nx + x) and link masks (bit i:
// link i pulls from, or passes through, a solid node of the body, or of a static wall).
struct LinkNode {
    size_t node;
    uint64_t body, wall;
};
void build_links(const HostLattice& H, int nx, int ny, const std::vector<uint8_t>& lab, std::vector<uint8_t>& cls,
                 std::vector<LinkNode>& links, size_t& n_fluid);
void constant_force(const HostLattice& H, const std::vector<LinkNode>& links, double rho0, double& fx, double& fy);
void tile_slots(int nx, int ny, int bx, int by, const std::vector<LinkNode>& links, std::vector<int>& slot, int& ntx,
                int& ntiles, int& nslots);
double drive_value(int drive, double u0, double omega, long n);
int fit_sincos(const double* fx, size_t stride, long n0, long n1, double omega, double coef[3]);

// What another translation unit may read of a simulation: its layout, tile shape and the launch
// parameters of its step kernel (device pointers to its geometry arrays included).
struct SimView {
    int device, Q, storage, collision, nx, ny, pitch, bx, by, nslots, drive;
    double u0, omega;
    InstDev inst;
    void* buf[2];
    int cur;
    long steps_done;
    double2* history;
    size_t esize, n_fluid;
    int aa;  // in-place single buffer (buf[1] is null)
    int variant;
    int ntiles;
    const CUtensorMap* maps;  // staged variants: load boxes of buf[0], buf[1]
};
SimView sim_view(const lbm_sim* s);
// Make room for `steps` entries of force history (may allocate).
int sim_reserve(lbm_sim* s, size_t steps);
// Store plain scaled deviations (no uniform-stream offset); only before the first step.
void sim_disable_stream_offset(lbm_sim* s);
// Record that `steps` steps were run on the simulation's buffers by another launcher.
void sim_advance(lbm_sim* s, long steps);
// The per-step constants (drive, 16-bit stream offsets) of the simulation's next `count` steps,
// exactly as lbm_step would set them.
void sim_step_constants(const lbm_sim* s, long count, StepConst* out);

}  // namespace lbm

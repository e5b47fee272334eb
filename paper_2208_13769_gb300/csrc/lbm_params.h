// lbm_params.h -- parameter blocks shared by the host library and the
// kernels of the fused Lagrangian LBM step (plain C++ structs, passed by
// value as kernel arguments or kept in device tables).
#pragma once

#include <stdint.h>

namespace lbm {

enum EdgeKind : int32_t { kPeriodic = 0, kDirichlet = 1, kNeumann = 2 };

// Layout of the state planes: node (x, y), x in [-3, nx + 3), y in [-3, ny + 3),
// sits at (y + kPadRows) * pitch + x + kPadCols.  Along a periodic axis the 3
// outer rows/columns hold images of the nodes across the seam; along a
// bounded axis the first ghost row/column holds the populations the boundary
// rules send back.  pitch is a multiple of 64 elements and kPadCols a
// multiple of 8, so every row segment the step kernel copies in bulk starts on
// a 16-byte boundary.
constexpr int kPadRows = 3;
constexpr int kPadCols = 8;

// One edge (0 = x-, 1 = x+, 2 = y-, 3 = y+) of Sec. 6's boundary value problem.
struct EdgeBC {
    int32_t kind;
    int32_t pad;
    double value[2];  // Dirichlet: u* at t = 0;  Neumann: T0
    double rate[2];   // Dirichlet: v*;           Neumann: T1
    double times[3];  // Neumann: t_on, t_ramp, t_off
};

struct StepParams {
    // geometry (see kPadRows / kPadCols)
    int32_t nx, ny;
    int32_t periodic_x, periodic_y;
    int64_t pitch;   // elements per row (storage or carry element type)
    int64_t plane;   // elements per plane
    int32_t scheme;  // 0 explicit (Algorithm 1), 1 predictor-corrector
    // interior kernel: output rectangle, its grid and its row ring
    int32_t rect[4];     // x_lo, x_hi, y_lo, y_hi
    int32_t tiles_x, tiles_y;  // column strips x row chunks
    int32_t chunk_rows;        // rows per chunk
    int32_t ring_slots;        // row slots of the bulk-copy ring (lookahead + 3)
    int32_t strip_x0;          // first column of strip 0
    int32_t strip_w;           // output columns per strip
    int32_t pad1[2];

    const void* f_src;  // 9 planes of f^col(t_n), storage type
    void* f_dst;        // 9 planes of f^col(t_n+1)
    const void* a_src;  // u-carry A: 2 components, in the layout of the format's carry type
    void* a_dst;
    const void* s_src;  // source carry 1S: 2 planes, arithmetic type
    void* s_dst;
    double* fields;      // NULL, or 5 planes [ny][nx] FP64: u_x, u_y, v_x, v_y, r
    const double* u0;    // init only: [ny][nx][2]
    const double* v0;    // init only: [ny][nx][2]
    int32_t* flag;       // bit 0: non-finite value or J <= 0 met
    int64_t* counter;    // two step counters (ping-pong by parity)
    int32_t parity;
    int32_t pad2;

    double dX, dt, c, cs2, omega, rho0, lambda, mu;
    double body[2];
    float enc_scale[9];  // 16-bit storage: 1 / (w_i 2^-s)
    float dec_scale[9];  // w_i 2^-s
    float lo_scale[2];   // u-carry with 16-bit low words: 2^k and 2^-k (UCompH)
    float pad3[2];
    EdgeBC bc[4];
    // lattice constants, computed once on the host in FP64 (kLat* indices);
    // lat_f holds the same values rounded to FP32
    double lat_d[16];
    float lat_f[16];
    // a rectangular hole (Sec. 7's plate with a hole): removed nodes x0 <= x
    // < x1, y0 <= y < y1 (x0 >= x1: none), and the constant traction on its
    // faces at x0, x1, y0, y1 (x and y components)
    int32_t hole[4];
    double hole_T[8];
};

// (x, y) is a removed node of the hole.
__host__ __device__ inline bool in_hole(const int32_t* h, int x, int y) {
    return x >= h[0] && x < h[1] && y >= h[2] && y < h[3];
}

// Indices into StepParams::lat_d / lat_f.
enum LatIndex : int {
    kLatOmega = 0,      // omega = dt / tau
    kLatOneMOmega,      // 1 - omega
    kLatForcePref,      // 1 - omega / 2
    kLatKu,             // dX / (2 rho0)
    kLatInv2dX,         // 1 / (2 dX)
    kLatSqScale,        // dt^2 / (2 dX^2)
    kLatSb0,            // (dt^2 / dX) rho0 b_x
    kLatSb1,            // (dt^2 / dX) rho0 b_y
    kLatLambda,         // lambda
    kLatMu,             // mu
    kLatInvC2,          // 1 / c^2
    kLatCOverRho0,      // c / rho0
    kLatRho0OverC,      // rho0 / c
    kLatRho0,           // rho0
    kLatCount
};

}  // namespace lbm

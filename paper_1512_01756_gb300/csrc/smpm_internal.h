// Internal declarations of libsmpm: host-side operator builders (host_ops.cpp),
// device kernels (kernels.cu) and the API / solve driver (api.cu).
#pragma once

#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/smpm.h"

namespace smpm {

// NVTX range for the lifetime of a scope (tracing: setups, solves and served
// batches show as named ranges in a profiler timeline; a no-op without one)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// Host side (plain C++, FP64)
// ---------------------------------------------------------------------------

// GLL points and quadrature weights on [-1, 1] (n points, order n-1).
void gll(int n, std::vector<double>& x, std::vector<double>& w);
// Nodal differentiation matrix, row-major n x n (D[i*n + j] = l_j'(x_i)).
void gll_diff(const std::vector<double>& x, std::vector<double>& D);

struct Geometry {
    int mx = 0, mz = 0, order = 0, n = 0, N = 0;
    int fz = 0, nx = 0;                   // z-nodes per strip column, x-nodes total
    long long r = 0, k = 0;               // grid nodes, Schur unknowns
    double lx = 0, lz = 0, hx = 0, tau_x = 0, z_ratio = 1, tau_scale = -0.1;
    std::vector<double> hz, zb, tau_z;    // per z-element
    std::vector<double> xi, w, D, D2;     // GLL data (row-major n x n)
    int ng = 1;                           // deflation groups per interface
    int d = 0;                            // coarse dimension (mx-1)*ng
};

// Fills every derived quantity; returns false on a bad argument (msg set).
bool make_geometry(int mx, int mz, int order, double lx, double lz, double z_ratio,
                   double tau_scale, int groups, Geometry& g, std::string& msg);

// 1-D x-operator of one strip class (n x n row-major): Laplacian plus the own
// part of the x-face terms (cls 0: Neumann west / Robin east, 1: Robin both,
// 2: Robin west / Neumann east).
void strip_x_operator(const Geometry& g, int cls, std::vector<double>& Ax);
// 1-D z-operator over the mz elements of a strip column (fz x fz row-major).
void z_operator(const Geometry& g, std::vector<double>& Lz);
// Full 1-D x-operator over all mx elements (nx x nx row-major) -- used only
// for the left null vector.
void full_x_operator(const Geometry& g, std::vector<double>& Lx);
// B-row coefficients of one strip class: beta[s*n + a], s = 0 for the flux
// written onto the west neighbour's east face, s = 1 onto the east neighbour's
// west face.  Zero rows where the class has no neighbour.
void face_flux_rows(const Geometry& g, int cls, std::vector<double>& beta);

// Banded LU with partial pivoting (column band storage, LAPACK layout).
struct BandLU {
    int n = 0, kl = 0, ku = 0, ldab = 0;
    std::vector<double> ab;
    std::vector<int> piv;
    void init(int n_, int kl_, int ku_);
    double& at(int i, int j) { return ab[(size_t)(kl + ku + i - j) + (size_t)j * ldab]; }
    double at(int i, int j) const { return ab[(size_t)(kl + ku + i - j) + (size_t)j * ldab]; }
    bool in_band(int i, int j) const { return i - j <= kl && j - i <= ku; }
    bool factor();                        // false if an exact zero pivot occurs
    void solve(double* b) const;          // A x = b  (in place)
    void solve_T(double* b) const;        // A^T x = b (in place)
};

// Unit left null vector of a dense-given banded singular matrix (row-major),
// by inverse iteration with (M - sigma I)^T.
bool left_null_banded(const std::vector<double>& M, int n, int bw, std::vector<double>& v,
                      std::string& msg);
// Unit left null vectors of the full 1-D x-operator (nx) and of the z-operator
// (fz); u_L = u_Lx (x) u_Lz is the left null vector of L (Kronecker sum).
bool left_null_x(const Geometry& g, std::vector<double>& v, std::string& msg);
bool left_null_z(const Geometry& g, std::vector<double>& v, std::string& msg);

// Coarse matrix of the deflation (d x d row-major, in place): for singular C
// (k^2 = 0, uC given) C + a uC 1^T / sqrt d, whose inverse times
// (I - uC uC^T) is the coarse division K (the zero-mean solution of the
// consistent coarse system); else C unchanged (K = C^-1).
void coarse_matrix(std::vector<double>& C, int d, int fz_over_ng, const double* uC);
bool tridiag_lu(int d, std::vector<double>& dl, std::vector<double>& dd, std::vector<double>& du,
                std::vector<double>& du2, std::vector<int>& swap);

// Ax = Q B Q^-1 with B block diagonal in real form: slot t covers columns
// [slot_start, slot_start + slot_size) of Q; size 1: eigenvalue alpha; size 2:
// the pair alpha +- i beta as the block [[alpha, beta], [-beta, alpha]].
bool real_block_diagonalise(const std::vector<double>& Ax, int n, std::vector<double>& Q, std::vector<double>& Qinv,
                            std::vector<int>& slot_start, std::vector<int>& slot_size, std::vector<double>& alpha,
                            std::vector<double>& beta, std::string& msg);

// ---------------------------------------------------------------------------
// Device side (kernels.cu)
// ---------------------------------------------------------------------------

// One tile of a class GEMM: columns c in [0, nu*nr) map to unit u0 + c / nr and
// right-hand side r0 + c % nr; every column of a tile uses matrix `mat`.
struct Tile {
    int mat, u0, nu, r0, nr;
    long long off;            // added to both the input and the output address
};

struct GemmArgs {
    const double* mats;       // matrix m at mats + m * mat_stride, row-major M x K
    long long mat_stride;
    int M, K;
    const int* row_lo;        // per matrix: output rows [row_lo, row_hi) are stored
    const int* row_hi;
    const double* in;         // column (u, r) at in + r*in_rs + u*in_us + in_off
    long long in_rs, in_us, in_off;
    double* out;              // row < msplit: out + r*out_rs + u*out_us + out_off0 + row
    long long out_rs, out_us, out_off0, out_off1;   // row >= msplit: ... + out_off1 + row - msplit
    int msplit;
    const double* add;        // EPI 1: out = add[same address] + acc
    const int* active;        // per rhs: skip tiles whose columns are all inactive (may be null)
    unsigned long long* flops;  // if set: each working CTA adds 2 * rows * K * active columns
    int fp32;                 // 1: mats are float, arithmetic in FP32 (EPI 0 only)
    double* out_lo;           // EPI 3: low parts of the compensated out = add + acc
    int shape;                // tile shape: 0 = 16 rows x 32 columns, 1 = 8 rows x 64 columns
    int mirror_nb;            // > 0: mirror form over columns of mirror_nb faces of `face` values;
                              // < 0: over -mirror_nb blocks of `face` values reversed inside each;
    int face;                 //   mats holds [Hp; Hm] (h x h each, h = M = K = |mirror_nb| face / 2)
};

// View of the operator data of operator set 0 that the allocation-free
// deflation projection (noalloc.cu) needs; filled by deflation_view (api.cu),
// which reads the handle only.
struct DeflView {
    int fz, mx, ng, d;
    long long k;
    const double* K;          // [d][d]
    const double* rho;        // [3 classes][2 sides][ng][2 fz]
    const int* strip_cls;     // [mx] (device)
    cudaStream_t stream;
};
bool deflation_view(smpm_handle h, DeflView* v, std::string& msg);
void set_last_error(const std::string& msg);

// Number of kernels libsmpm has launched in this process.
long long launch_count();
void count_launches(int n);

void launch_class_gemm(const GemmArgs& a, const Tile* d_tiles, int ntiles, int epi, void* stream);
// columns per tile of a tile shape (the tile lists of a launch are built for it)
int gemm_tile_columns(int shape);

// Describes the vector batch layout shared by the small kernels.
struct VecLayout {
    int R;                    // right-hand sides in the batch
    long long ld;             // stride between the face vectors of consecutive rhs
    long long kp;             // padded face-vector length (2 fz mx)
    int fz, mx, ng, d, n;
};

}  // namespace smpm

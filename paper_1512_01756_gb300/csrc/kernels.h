// Launch wrappers of the libsmpm device kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "smpm_internal.h"

namespace smpm {

// Face-vector layout: for strip i, face s (0 = west, 1 = east) the fz values
// sit at offset (2 i + s) fz of a padded vector of length kp = 2 fz mx; the
// two physical faces (strip 0 west, strip mx-1 east) are padding and hold 0.
// Interface t (between strips t and t+1) is the contiguous range
// [(2 t + 1) fz, (2 t + 3) fz).  ld >= kp + fz is the stride between the
// vectors of consecutive right-hand sides.

// Per-solve arguments of the Krylov / deflation kernels.
struct KArgs {
    int R, m, nch, ch;             // rhs, restart length, chunks, chunk length
    long long ld, kp;
    int fz, mx, ng, d, n;
    double* V;                     // [R][m+1][ld]  Arnoldi basis
    double* w;                     // [R][ld]       work vector
    double* Hc;                    // [R][m][m+1]   rotated Hessenberg columns
    double* htmp;                  // [R][m+1]      first CGS pass coefficients
    double* cs;                    // [R][m]        Givens cosines
    double* sn;                    // [R][m]        Givens sines
    double* gv;                    // [R][m+1]      rotated residual vector
    double* part1;                 // [R][nch][m+2] partial dot products
    double* part2;
    double* q;                     // [R][d]        coarse restriction Z^T v
    double* c;                     // [R][d]        coarse solution K q
    const double* rho;             // op o: rho + o*rho_stride, [cls][side][ng][2 fz]
    long long rho_stride;
    const double* K;               // op o: K + o*K_stride, [d][d]; null: no deflation (c = 0)
    long long K_stride;
    const int* op;                 // [R] operator set of each rhs
    const int* strip_cls;          // [mx]
    int* active;                   // [R] running Arnoldi in this cycle
    int* done;                     // [R] converged (or stopped)
    int* nit;                      // [R] Arnoldi steps taken in this cycle
    double* target;                // [R] absolute residual target tol*||b_S||
    double* bnorm;                 // [R] ||b_S||
    double* rnorm;                 // [R] residual norm at the last cycle start
    int* flags;                    // [R] bit 0: breakdown / non-finite
    // extended-precision refinement (all null when off): x_S = xS + xlo, and
    // S x_S = s + s_lo + s_xlo (compensated S xS, plain S xlo)
    double* xlo;                   // [R][ld]
    const double* s_lo;            // [R][ld]
    const double* s_xlo;           // [R][ld]
    // right-hand sides per Krylov space: 1 = one space per column; grp > 1:
    // columns [g grp, (g+1) grp) form one concatenated vector (Sec. 5: all
    // wavenumbers in one GMRES), every dot product and norm summed over them
    int grp;
    // 1: the CGS2 projections and dot products in FP32 arithmetic on the FP64
    // vectors (the inner solve of the nested mixed-precision form, which only
    // has to reach 1e-4 and whose Arnoldi work is bound by the FP64 pipe)
    int f32;
    // residual history (null: off): hist[r * hist_stride + hist_base[r] + j + 1]
    // = |Givens residual| / ||b_S|| after Arnoldi step j of the current cycle
    double* hist;
    const int* hist_base;
    int hist_stride;
};

void k_deflate_sum(const KArgs& a, const double* v, const double* vsub, cudaStream_t s);
void k_coarse(const KArgs& a, cudaStream_t s);
// mode 0: w -= S Z c, dots with V[0..j];  mode 1: reduce pass 1, w -= V h1, dots;
// mode 2: reduce pass 2, w -= V h2, store Hessenberg column, partial norms.
void k_cgs(const KArgs& a, int j, int mode, cudaStream_t s);
// beta = ||w||, V[j+1] = w / beta, Givens update, convergence flags.
void k_normalize(const KArgs& a, int j, int last_allowed, cudaStream_t s);
// Start of a restart cycle (iterative refinement on x_S): d = b_S - s with
// s = S x_S (null on the first cycle), q = Z^T d, c = K q, V[0] = P d = d - S Z c,
// partial norms ||P d||, ||b_S||, ||d||; then k_cycle_start tests ||d|| against
// tol ||b_S||, normalises V[0] and saves c into c0.
void k_residual(const KArgs& a, const double* bS, const double* sv, cudaStream_t s);
void k_cycle_start(const KArgs& a, double* c0, int first, double tol, cudaStream_t s);
// Y = basis y with y from the rotated Hessenberg system of the cycle (basis:
// the Arnoldi vectors V by default, or the preconditioned vectors of FGMRES).
void k_cycle_update(const KArgs& a, double* Y, cudaStream_t s, const double* basis = nullptr,
                    long long basis_rs = 0);
// c = K Z^T v for every unconverged rhs.
void k_deflate_coarse_pending(const KArgs& a, const double* v, cudaStream_t s);
// x_S += t + Z (c0 - c) for rhs that ran this cycle.
void k_xs_update(const KArgs& a, double* xS, const double* t, const double* c0, cudaStream_t s);

// One dense-product launch as the persistent Arnoldi kernel runs it: the
// GEMM arguments, the device tile list of the chosen tile shape (a.shape)
// and the launch's column tiles and row tiles; a.mirror_nb != 0 selects the
// mirror form.
struct PGemm {
    GemmArgs a;
    const Tile* tiles;
    int ntiles, nrow;
    int epi;                       // 0: store, 1: add a.add
};

// The Arnoldi steps j0 .. last_allowed-1 of one restart cycle for every
// active right-hand side in one cooperative launch (Sec. 3, Alg. seq step 4:
// block-Jacobi apply, Schur product, deflation, CGS2, normalisation and
// Givens per step), the phases separated by grid-wide barriers.
struct PersistArgs {
    KArgs ka;
    PGemm bj[2][2];                // block-Jacobi launches: [0] FP64 blocks, [1] FP32 blocks
    int nbj[2];
    PGemm sc[2];                   // Schur product launches
    int nsc;
    long long bj_step;             // block-Jacobi input offset per step (the basis slot stride)
    int j0, last_allowed;
    int fp64_steps;                // steps j < fp64_steps use the FP64 blocks
    int use_fp32;                  // steps from fp64_steps on use the FP32 blocks
    double* Zb;                    // flexible GMRES: z_j kept at Zb + r*m*ld + j*ld (null: off)
    const double* z;               // the block-Jacobi output z_j ([R][ld])
    unsigned int* bar;             // barrier counter, zero at launch
    int* status;                   // set to 1 by a barrier wait that ran out of time
    long long wait_ns;             // time limit of one barrier wait
    int stall;                     // test hook: every barrier waits for one block more than the grid has
};
// Launch the persistent kernel on `s` (cooperative launch, as many blocks as
// fit on the device); false if the device cannot launch it cooperatively.
bool k_arnoldi_persistent(const PersistArgs& p, cudaStream_t s);

// FP64-accurate class GEMM on the tensor cores (ozaki.cu): the class
// matrices pre-split into S BF16 digit matrices of beta bits (row scale
// 2^rexp), the input columns split on the fly, anti-diagonal digit products
// accumulated exactly in FP32 tensor memory and combined in 64-bit integers.
struct OzArgs {
    GemmArgs a;                    // columns, addressing, rows, epilogue as for the class GEMM (mats unused)
    const unsigned short* dig;     // matrix m: dig + m * dig_stride, [mt_n][kcn][S][128 x 128] digit blocks
    long long dig_stride;
    const int* rexp;               // matrix m: rexp + m * rexp_stride, [mt_n * 128] row exponents
    long long rexp_stride;
    int S, beta, N, mt_n, kcn, epi;
    int* err;                      // set to 2 by a wait that ran out of iterations
};
// beta, S and the column-tile width N for inner dimension K (false: K too large)
bool oz_choose(int K, int& S, int& beta, int& N, int bits = 56);
int oz_smem_bytes(int S, int N);
void k_oz_split_rows(const double* mats, long long mat_stride, int nmat, int M, int K, int S, int beta, int mt_n,
                     int kcn, unsigned short* dig, long long dig_stride, int* rexp, long long rexp_stride,
                     cudaStream_t s);
void k_oz_split_rows_f(const float* mats, long long mat_stride, int nmat, int M, int K, int S, int beta, int mt_n,
                       int kcn, unsigned short* dig, long long dig_stride, int* rexp, long long rexp_stride,
                       cudaStream_t s);
// false if the launch could not be configured (shared-memory limit)
bool launch_oz_gemm(const OzArgs& z, const Tile* d_tiles, int ntiles, cudaStream_t s);

// RHS assembly b = f + tau g at the physical boundary, per rhs; partial
// dots with u_L for the projection (uL[r] may be null).
struct GridArgs {
    int n, N, mx, mz, fz, nx;
    long long r;
    double tau_x;
    const double* tau_z;           // [mz] (device)
    const double* wq;              // [n] GLL weights (device)
    const double* hz;              // [mz] (device)
    double hx, area;
};
void k_rhs_assemble(const GridArgs& g, int R, const double* f, long long f_ld, const double* gb,
                    long long g_ld, double* b, long long b_ld, const double* const* uL,
                    double* part, int nch, int ch, cudaStream_t s);
void k_project(int R, long long len, double* v, long long v_ld, const double* const* u,
               const double* part, int nch, int ch, cudaStream_t s);
void k_dot_partial(int R, long long len, const double* v, long long v_ld, const double* const* u,
                   double* part, int nch, int ch, cudaStream_t s);
void k_recovery_rhs(const GridArgs& g, int R, const double* b, long long b_ld, const double* xS,
                    long long x_ld, double* t2, cudaStream_t s);
void k_gauge(const GridArgs& g, int R, double* u, long long u_ld, const int* apply, double* part,
             int nch, int ch, cudaStream_t s);

// Setup builders.
void k_build_strip_op(double* A, const double* Ax, const double* Lz, double k2, int n, int fz,
                      cudaStream_t s);
void k_identity(double* X, int m, cudaStream_t s);
// per matrix: |A v - fl32(B) v| / |A v| for a fixed sign vector (FP32 copy adequacy)
void k_fp32_quality(const double* A, const float* B, int m, long long stride, int nmat, double* out, cudaStream_t s);
// real DFT along y: [my][n] -> [my/2+1][2][n] (scaled by 1/my) and back; cs = [cos; sin](2 pi idx / my)
void k_dft_forward(const double* in, double* out, const double* cs, long long n, int my, cudaStream_t s);
void k_dft_inverse(const double* in, double* out, const double* cs, long long n, int my, cudaStream_t s);
// dst = P src P, P reversing the nb face blocks of an (nb fz)^2 matrix (mirror image)
void k_mirror_blocks(double* dst, const double* src, int fz, int nb, cudaStream_t s);
// Mirror symmetry of a class matrix (nb = 2 or 4 faces of fz values, J the
// reversal of the face order): res[0] = max |Mat - J Mat J|, res[1] = max |Mat|.
void k_mirror_asym(const double* Mat, int fz, int nb, double* res, cudaStream_t s);
// Mat <- (Mat + J Mat J) / 2 in place.
void k_mirror_symmetrize(double* Mat, int fz, int nb, cudaStream_t s);
// The two h x h halves of the mirror form, H = [Hp; Hm] (h = nb fz / 2):
// Hp, Hm = (Mat[i][j] +- Mat[i][mirror(j)]) / 2 for i, j < h.
void k_mirror_halves(double* H, const double* Mat, int fz, int nb, cudaStream_t s);
void k_mirror_halves_f(float* H, const float* Mat, int fz, int nb, cudaStream_t s);
// Halves of count slot matrices (nblk blocks of fz values, fz even, stride
// (nblk fz)^2) under the z-reversal inside each block: H[c] = [Hp; Hm].
// done[r] = active[r] ? 0 : 1 for r < R
void k_invert_flags(int* done, const int* active, int R, cudaStream_t s);
// K <- K - (K u) u^T (row-major d x d, w: d scratch): the projected coarse division
void k_project_coarse(double* K, double* w, const double* u, int d, cudaStream_t s);
void k_tridiag_inverse(double* K, const double* fac, const int* swap, int d, cudaStream_t s);
void k_build_W(double* W, const double* Ainv, const double* beta, int n, int fz, cudaStream_t s);
void k_build_G(double* G, const double* W, int n, int fz, int cls, cudaStream_t s);
// Pair block of block-Jacobi (Sec. 3.2) from the G of strips 2p, 2p+1, 2p+2
// (gC null for the single-interface last block).
void k_build_M(double* M, const double* gA, const double* gB, const double* gC, int fz,
               cudaStream_t s);
void k_pad_block(double* dst, const double* src, int m_src, int m_dst, cudaStream_t s);
void k_build_rho(double* rho, const double* G, int fz, int ng, cudaStream_t s);
void k_fill(double* x, long long n, double v, cudaStream_t s);
void k_to_fp32(float* dst, const double* src, long long n, cudaStream_t s);
void k_identity_f(float* X, int m, cudaStream_t s);
void k_pad_block_f(float* dst, const float* src, int m_src, int m_dst, cudaStream_t s);

// Fast strip solver pieces.
struct FssArgs {
    int n, fz, nstrips;
    const int* cls;                // [nstrips] class of each strip (device)
};
// out[r][strip][a][Z] = sum_b T_cls[a][b] (in[r][strip][b][Z] - (E x_S)[...]);
// T holds the 3 class matrices [3][n][n]; xS (face layout) may be null.
void k_xform(const FssArgs& f, int R, const double* T, const double* in, long long in_ld, double* out,
             long long out_ld, const double* xS, long long x_ld, cudaStream_t s, const double* addv = nullptr,
             long long add_ld = 0);
// res = (b - E x_S) - A_c(k) x per strip (k^2 per right-hand side in k2r).
void k_strip_residual(const FssArgs& f, int R, const double* Ax3, const double* Lz, const int* zlo, const int* zhi,
                      const double* k2r, const double* b, long long b_ld, const double* xS, long long x_ld,
                      const double* x, long long xv_ld, double* res, long long r_ld, cudaStream_t s);
// b_S = B y on the padded face layout (beta: [3][2][n]).
void k_face_flux(const FssArgs& f, int R, const double* beta, const double* y, long long y_ld, double* bS,
                 long long b_ld, long long kp, cudaStream_t s);
void k_build_slot(double* M, const double* Lz, int fz, int size, double shift, double beta, cudaStream_t s);
void k_build_slot_halves(double* H, const double* Lz, int fz, int size, double shift, double beta, cudaStream_t s);
// Batched Gauss-Jordan inversion with partial pivoting, one CTA per matrix
// (row-major n x n, src and dst device arrays of count pointers; info[b] != 0:
// zero or non-finite pivot).  Shared memory up to n = gj_smem_max().
void k_gj_inverse(const double* const* src, double* const* dst, int n, int count, int* info, cudaStream_t s);
int gj_smem_max();
void k_unit_faces(double* U, int n, int fz, cudaStream_t s);
void k_g_from_solves(double* G, const double* Y, const double* beta, int n, int fz, int cls, cudaStream_t s);

// FP64 DFMA throughput probe: each thread runs `iters` dependent-chain-free
// FMA groups; returns nothing, writes a checksum to out.
void k_fp64_probe(double* out, int blocks, int iters, cudaStream_t s);

}  // namespace smpm

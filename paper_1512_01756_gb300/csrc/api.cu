// libsmpm: handle, operator setup and the batched solve driver behind the C ABI
// of include/smpm.h.
//
// Setup (Secs. 2.3, 3.2, 3.3, 5): for every strip class c (west boundary,
// interior, east boundary) and every k^2 of the handle the dense strip operator
// A_c(k) = Ax_c (+) L_z - k^2 I is LU-factored (cuSOLVER getrf/getrs, setup
// only) into an explicit inverse; W_c = B_c A_c^-1 (right-hand-side map),
// G_c = W_c E_c (Schur blocks), the block-Jacobi pair blocks and their
// inverses, the row sums rho_c of G_c that give S Z, the coarse operator K and,
// for k^2 = 0, the null vectors u_L = u_Lx (x) u_Lz and u_S = E^T u_L (Claim 1).
//
// Solve (Alg. seq): b = f + tau g, b <- b - u_L u_L^T b, b_S = W b,
// b_S <- b_S - u_S u_S^T b_S, right-preconditioned deflated GMRES on
// P S M^-1 y = P b_S with CGS2 Arnoldi and restarts, x_S = t + Z K Z^T (b_S - S t)
// with t = M^-1 y (= Q M^-1 y + Z C\(...) b_S), recovery u = A^-1 (b - E x_S),
// zero-mean gauge for k^2 = 0.  Every step runs in kernels.cu; the host only
// sequences launches and reads convergence flags.
#include <cuda_runtime.h>
#include <cusolverDn.h>
#include <cublas_v2.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/smpm.h"
#include "kernels.h"
#include "smpm_internal.h"

namespace smpm {

static thread_local std::string g_last_error;

struct Err {
    int code;
    std::string msg;
};

#define CK(x)                                                                              \
    do {                                                                                   \
        cudaError_t e_ = (x);                                                              \
        if (e_ != cudaSuccess) throw Err{SMPM_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)}; \
    } while (0)
#define CS(x)                                                                              \
    do {                                                                                   \
        cusolverStatus_t s_ = (x);                                                         \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                                 \
            throw Err{SMPM_ECUDA, std::string(#x) + ": cusolver status " + std::to_string((int)s_)}; \
    } while (0)

// Tile lists of one GEMM site, built for both tile shapes (0: 16 x 32,
// 1: 8 x 64; columns per tile gemm_tile_columns(shape)).
struct TileSet {
    Tile* t[2] = {nullptr, nullptr};
    int n[2] = {0, 0};
    size_t cap = 0;
};
static constexpr int kChunk = 1024; // vector-kernel chunk

struct Solver {
    Geometry g;
    smpm_grid opt{};
    cudaStream_t stream = nullptr;
    int nop = 1;
    std::vector<double> k2;
    int singular_op = -1;
    int P = 0, nmc = 0;                      // block-Jacobi blocks and block classes
    std::vector<int> strip_cls, pair_mc, mc_single;
    long long kp = 0, ld = 0;
    int restart = 64, max_iter = 2000;
    // fast strip solver (x-factor block diagonalisation; see kernels.cu)
    bool fss = false;
    double *d_Q = nullptr, *d_Qinv = nullptr, *d_beta = nullptr;   // [3][n][n], [3][n][n], [3][2][n]
    std::vector<int> sl_start[3], sl_size[3], sl_idx[3];             // per class: slot start, size, index in its size list
    int ns1 = 0, ns2 = 0;                                            // max size-1 / size-2 slots over the classes
    double *S1 = nullptr, *S2 = nullptr;                             // slot inverses [nop][3][ns][m*m]
    bool zmir = false;                                               // slots in the z-mirror form
    double *S1h = nullptr, *S2h = nullptr;                           // their halves [nop][3][ns][2][(m/2)^2]
    int *rl_S1 = nullptr, *rh_S1 = nullptr, *rl_S2 = nullptr, *rh_S2 = nullptr;
    int* d_cls3 = nullptr;                                           // {0, 1, 2}
    double *d_Ax3 = nullptr, *d_Lz = nullptr;                        // x-factors [3][n][n], z-operator [fz][fz]
    int *d_zlo = nullptr, *d_zhi = nullptr;                          // nonzero window of each L_z row
    // device operators (all ops, contiguous per kind)
    double *Ainv = nullptr, *W = nullptr, *G = nullptr, *Minv = nullptr, *rho = nullptr, *K = nullptr;
    float* Minv32 = nullptr;              // FP32 block-Jacobi inverses (precision 1 and 2)
    float* G32 = nullptr;                 // FP32 Schur blocks (precision 2: the inner solve)
    double fp32_err = 0.0;                // measured relative error of the FP32 block-Jacobi apply
    bool bj32_ok = true;                  // FP32 blocks adequate (precision 1 uses them)
    int inner_m = 10;                     // inner Arnoldi steps per outer step (precision 2)
    // physical-space 3-D solve (handles from smpm_setup_3d)
    int my = 0;
    double* d_cs = nullptr;               // [cos; sin](2 pi idx / my)
    double *f3hat = nullptr, *g3hat = nullptr, *u3hat = nullptr, *f3stage = nullptr;
    long long cap3 = 0, capg3 = 0;
    int precision = 0;
    int krylov = 0;                       // 1: one concatenated Krylov space per solve call
    double *uL = nullptr, *uS = nullptr;
    double* oneS = nullptr;                 // right null vector of S(0): 1 on the interface faces, unit norm
    int *rl_GW = nullptr, *rh_GW = nullptr, *rl_M = nullptr, *rh_M = nullptr, *rl_A = nullptr, *rh_A = nullptr;
    int* d_strip_cls = nullptr;
    double *d_tau_z = nullptr, *d_wq = nullptr, *d_hz = nullptr;
    long long sA = 0, sW = 0, sG = 0, sM = 0, sRho = 0, sK = 0;
    // workspace
    int Rcap = 0;
    struct Work {
        double *b = nullptr, *t2 = nullptr, *bS = nullptr, *Xp = nullptr, *t = nullptr, *s = nullptr;
        double *w = nullptr, *z = nullptr, *xS = nullptr, *V = nullptr;
        double *xSlo = nullptr, *slo = nullptr, *sxlo = nullptr;   // extended-precision refinement
        // inner FP32-operator DBJ-GMRES of the nested mixed-precision form (precision 2)
        double *Vi = nullptr, *Hci = nullptr, *htmpi = nullptr, *csi = nullptr, *sni = nullptr, *gvi = nullptr;
        double *part1i = nullptr, *part2i = nullptr, *qi = nullptr, *ci = nullptr, *c0i = nullptr;
        double *targeti = nullptr, *bnormi = nullptr, *rnormi = nullptr;
        double *wi = nullptr, *zi = nullptr, *xi = nullptr, *ti = nullptr, *si = nullptr, *Xpi = nullptr, *vin = nullptr;
        int *activei = nullptr, *donei = nullptr, *niti = nullptr, *flagsi = nullptr;
        double *Hc = nullptr, *htmp = nullptr, *cs = nullptr, *sn = nullptr, *gv = nullptr;
        double *part1 = nullptr, *part2 = nullptr, *q = nullptr, *c = nullptr, *c0 = nullptr;
        double *fstage = nullptr, *gstage = nullptr, *ustage = nullptr, *rpart = nullptr;
        int *active = nullptr, *done = nullptr, *nit = nullptr, *flags = nullptr, *op = nullptr, *gauge = nullptr;
        double *target = nullptr, *bnorm = nullptr, *rnorm = nullptr;
        const double** uLp = nullptr;
        const double** uSp = nullptr;
        const double** oneSp = nullptr;
        TileSet tM, tG, tW, tA, tS1, tS2;
        TileSet tGb, tGm, tMb, tMm;       // boundary-class / mirror-form tiles
        double *fs1 = nullptr, *fs2 = nullptr, *fs3 = nullptr, *k2r = nullptr;
        double* Zb = nullptr;             // FGMRES preconditioned vectors [R][m][ld] (precision 1)
        double* hist = nullptr;           // [R][max_iter + 1] Givens residual estimates per Arnoldi step
        int* hist_base = nullptr;         // [R] steps before the current cycle
        std::vector<void*> allocs;
    } wk;
    // residual history of the last solve: per right-hand side, the relative
    // true residual at every cycle start (host), and the number of Arnoldi
    // steps whose Givens estimates are in wk.hist
    std::vector<std::vector<double>> hist_true;
    std::vector<int> hist_steps;
    int hist_R = 0;
    std::vector<int> cur_ops;               // op layout the tiles were built for
    std::vector<void*> allocs;
    long long bytes = 0, wk_bytes = 0;
    std::vector<double> last_res;           // per-rhs ||S x_S - b_S|| / ||b_S|| of the last solve
    double setup_ms = 0.0;
    cusolverDnHandle_t sol = nullptr;
    int slot_cls[3] = {0, 1, 2};            // class whose slot inverses a class uses (mirror sharing)
    // Mirror form of the interior Schur blocks and block-Jacobi pairs (uniform
    // h_x): halves [Hp; Hm] per operator, FP64 and FP32 copies
    bool mirG = false, mirM = false;        // halves built
    bool useG = false, useM = false;        // used by the current batch (prepare_ops)
    int mirror_mode = 2;                    // SMPM_MIRROR at setup: 0 off, 1 always, 2 by size
    int mc_int = -1;                        // block class of the interior pairs
    double *Gh = nullptr, *Mh = nullptr;
    float *Gh32 = nullptr, *Mh32 = nullptr;
    // optional profiling of the class-GEMM launches (events + device flop counter)
    // CUDA graphs of the Arnoldi step groups (between two convergence checks),
    // keyed by (first step, steps, steps allowed in the cycle); valid for the
    // current workspace, operator layout and profiling state.  A group is
    // captured the second time it runs with the same key and replayed after.
    struct GroupGraph {
        cudaGraphExec_t exec = nullptr;
        long long launches = 0;              // library kernels in the graph
        std::vector<cudaEvent_t> ev;         // GEMM event pairs (profiling)
        std::vector<char> f32;               // 1 for an FP32 launch, per event pair
    };
    std::map<std::array<int, 4>, GroupGraph> graphs;
    std::map<std::array<int, 4>, int> group_seen;
    cudaStream_t cap_stream = nullptr;
    std::vector<cudaEvent_t>* cap_events = nullptr;   // set while capturing with profiling on
    std::vector<char>* cap_f32 = nullptr;
    bool graphs_ok = true;
    // persistent Arnoldi kernel: barrier counter and status word (device),
    // off for the handle once a cooperative launch has been refused
    bool persist_ok = true;
    // FP64-accurate tensor-core products (ozaki.cu): digit tensors of the
    // Schur blocks G and the block-Jacobi inverses, keyed by the FP64 matrix
    // array they were split from
    struct OzMat {
        unsigned short* dig = nullptr;
        int* rexp = nullptr;
        long long dig_stride = 0, rexp_stride = 0;
        int S = 0, beta = 0, N = 0, mt_n = 0, kcn = 0;
    };
    bool oz = false;
    int oz_mask = 0;                      // 1: FP64 products, 2: FP32 products on the tensor cores
    std::map<const double*, OzMat> ozmats;
    int* d_ozerr = nullptr;
    unsigned int* d_pbar = nullptr;
    int* d_pstatus = nullptr;
    bool capturing = false;
    // profiled launches inside a graph capture take the CUDA-core path, whose
    // event bookkeeping handles captures
    bool capturing_prof_block() const { return prof && cap_events != nullptr; }                 // a group is being captured (no tuning, no syncs)
    void drop_graphs() {
        for (auto& kv : graphs) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            for (cudaEvent_t e : kv.second.ev) cudaEventDestroy(e);
        }
        graphs.clear();
        group_seen.clear();
    }
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    std::vector<char> ev_f32;               // category of each recorded launch (0 FP64, 1 FP32, 2 tensor)
    int ev_used = 0;
    unsigned long long* d_flops = nullptr;  // [0] FP64 launches, [1] FP32 launches
    // per category: 0 FP64 CUDA-core products, 1 FP32 products, 2 FP64-accurate
    // tensor-core products (algorithmic FLOPs), 3 the same launches' executed
    // BF16 tensor FLOPs (time counted under 2)
    long long prof_launches[4] = {0, 0, 0, 0};
    double prof_ms[4] = {0.0, 0.0, 0.0, 0.0}, prof_flops[4] = {0.0, 0.0, 0.0, 0.0};

    template <class T>
    T* dalloc(size_t n, std::vector<void*>& list) {
        void* p = nullptr;
        if (n == 0) n = 1;
        // stream-ordered: no device-wide synchronisation, so handles on other
        // streams (the serving workers) keep running while this one allocates
        cudaError_t e = cudaMallocAsync(&p, n * sizeof(T), stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Err{SMPM_ENOMEM, std::string("device allocation of ") + std::to_string(n * sizeof(T)) +
                                       " bytes failed: " + cudaGetErrorString(e)};
        }
        list.push_back(p);
        bytes += (long long)(n * sizeof(T));
        return (T*)p;
    }
    void free_list(std::vector<void*>& list) {
        for (void* p : list) cudaFreeAsync(p, stream);
        list.clear();
    }
    ~Solver() {
        if (stream) cudaStreamSynchronize(stream);
        drop_graphs();
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        free_list(wk.allocs);
        free_list(allocs);
        if (stream) cudaStreamSynchronize(stream);
        if (sol) cusolverDnDestroy(sol);
    }
};

// ---------------------------------------------------------------------------
// Setup
// ---------------------------------------------------------------------------

static void upload(double* dst, const std::vector<double>& src, cudaStream_t s) {
    CK(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice, s));
}

// dst <- src^-1 for an m x m row-major matrix in device memory (src is destroyed).
static void invert_dense(Solver& S, double* src, double* dst, int m, double* work, int lwork, int* ipiv, int* info) {
    // cuSOLVER is column-major: the row-major buffer is read as src^T; solving
    // src^T X = I in column-major gives X = src^-T, i.e. src^-1 in row-major.
    k_identity(dst, m, S.stream);
    CS(cusolverDnDgetrf(S.sol, m, m, src, m, work, ipiv, info));
    CS(cusolverDnDgetrs(S.sol, CUBLAS_OP_N, m, m, src, m, ipiv, dst, m, info));
    int h_info = 0;
    CK(cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, S.stream));
    CK(cudaStreamSynchronize(S.stream));
    if (h_info != 0) throw Err{SMPM_EBREAKDOWN, "singular strip or block-Jacobi matrix (getrf info " + std::to_string(h_info) + ")"};
}

static void run_gemm(Solver& S, GemmArgs a, const TileSet& ts, int epi);

// Fast strip solve out = A_c(k)^-1 (in - E x_S) on nstrips strips (classes in fa.cls)
// for R right-hand sides: x-transform by Q^-1, the slot inverses of B_c (+) L_z - k^2
// (class GEMMs over the size-1 and size-2 slots), x-transform by Q.
static void fss_run(Solver& S, const FssArgs& fa, int R, const double* in, long long in_ld, double* out,
                    long long out_ld, const double* xS, long long x_ld, double* t1, double* t2, const TileSet& tS1,
                    const TileSet& tS2, bool accumulate = false) {
    const int fz = S.g.fz, n = S.g.n;
    const long long nfz = (long long)n * fz, ld = (long long)fa.nstrips * nfz;
    k_xform(fa, R, S.d_Qinv, in, in_ld, t1, ld, xS, x_ld, S.stream);
    for (int sz = 1; sz <= 2; ++sz) {
        GemmArgs a;
        std::memset(&a, 0, sizeof(a));
        a.mats = sz == 1 ? S.S1 : S.S2;
        a.mat_stride = (long long)sz * fz * sz * fz;
        a.M = a.K = sz * fz;
        a.row_lo = sz == 1 ? S.rl_S1 : S.rl_S2;
        a.row_hi = sz == 1 ? S.rh_S1 : S.rh_S2;
        a.in = t1; a.in_rs = ld; a.in_us = nfz; a.in_off = 0;
        a.out = t2; a.out_rs = ld; a.out_us = nfz; a.out_off0 = 0; a.out_off1 = 0; a.msplit = sz * fz;
        if (S.zmir) {   // z-mirror form of the slot products
            const int h = sz * fz / 2;
            a.mats = sz == 1 ? S.S1h : S.S2h;
            a.mat_stride = 2LL * h * h;
            a.M = a.K = h;
            a.mirror_nb = -sz;
            a.face = fz;
        }
        run_gemm(S, a, sz == 1 ? tS1 : tS2, 0);
    }
    k_xform(fa, R, S.d_Q, t2, ld, out, out_ld, nullptr, 0, S.stream, accumulate ? out : nullptr, out_ld);
}

// Fast strip solve with one step of iterative refinement: x0 = FSS(b - E x_S),
// res = (b - E x_S) - A_c(k) x0 in FP64 through the Kronecker-sum structure,
// out = x0 + FSS(res).  The slot inverses (L_z + (alpha - k^2) I)^-1 are
// individually ill-conditioned (~1e6), so one unrefined pass is accurate to
// ~1e-10 only; the refined result matches a dense LU solve (~1e-13).
static void fss_refined(Solver& S, const FssArgs& fa, int R, const double* in, long long in_ld, double* out,
                        long long out_ld, const double* xS, long long x_ld, const double* k2r, double* t1, double* t2,
                        double* t3, const TileSet& tS1, const TileSet& tS2) {
    const long long ld = (long long)fa.nstrips * S.g.n * S.g.fz;
    fss_run(S, fa, R, in, in_ld, out, out_ld, xS, x_ld, t1, t2, tS1, tS2);
    k_strip_residual(fa, R, S.d_Ax3, S.d_Lz, S.d_zlo, S.d_zhi, k2r, in, in_ld, xS, x_ld, out, out_ld, t3, ld, S.stream);
    fss_run(S, fa, R, t3, ld, out, out_ld, nullptr, 0, t1, t2, tS1, tS2, true);
}

// Slot tiles of one class on a single strip: operators o0 .. o0 + no - 1,
// Rper right-hand sides each (operator o0 + q owns columns [q Rper, (q+1) Rper)).
static std::vector<Tile> single_strip_slot_tiles(const Solver& S, int o0, int no, int c, int Rper, int sz, int bn) {
    std::vector<Tile> out;
    const int ns = std::max(sz == 1 ? S.ns1 : S.ns2, 1);
    for (int q = 0; q < no; ++q)
        for (size_t t = 0; t < S.sl_size[c].size(); ++t) {
            if (S.sl_size[c][t] != sz) continue;
            for (int rr = 0; rr < Rper; rr += bn)
                out.push_back(Tile{((o0 + q) * 3 + S.slot_cls[c]) * ns + S.sl_idx[c][t], 0, 1, q * Rper + rr,
                                   std::min(bn, Rper - rr), (long long)S.sl_start[c][t] * S.g.fz});
        }
    return out;
}

// A_c(k)^-1 of strip vectors of class c for setup: Rper right-hand sides for
// each of the operators o0 .. o0 + no - 1, all in one refined fast solve.
static void fss_setup(Solver& S, int o0, int no, int c, int Rper, const double* in, double* out, double* t1,
                      double* t2, std::vector<void*>& tmp) {
    FssArgs fa{S.g.n, S.g.fz, 1, S.d_cls3 + c};
    const int R = no * Rper;
    TileSet ts[2];
    std::vector<Tile> tv[2][2];
    for (int sz = 1; sz <= 2; ++sz)
        for (int sh = 0; sh < 2; ++sh) {
            tv[sz - 1][sh] = single_strip_slot_tiles(S, o0, no, c, Rper, sz, gemm_tile_columns(sh));
            const auto& v = tv[sz - 1][sh];
            ts[sz - 1].t[sh] = S.dalloc<Tile>(std::max<size_t>(v.size(), 1), tmp);
            ts[sz - 1].n[sh] = (int)v.size();
            if (!v.empty())
                CK(cudaMemcpyAsync(ts[sz - 1].t[sh], v.data(), v.size() * sizeof(Tile), cudaMemcpyHostToDevice, S.stream));
        }
    const long long nfz = (long long)S.g.n * S.g.fz;
    std::vector<double> k2h((size_t)R);
    for (int r = 0; r < R; ++r) k2h[r] = S.k2[o0 + r / Rper];
    double* k2r = S.dalloc<double>((size_t)R, tmp);
    upload(k2r, k2h, S.stream);
    double* t3 = S.dalloc<double>((size_t)R * nfz, tmp);
    fss_refined(S, fa, R, in, nfz, out, nfz, nullptr, 0, k2r, t1, t2, t3, ts[0], ts[1]);
    CK(cudaStreamSynchronize(S.stream));
}

// Setup lanes: extra streams, each with its own cuSOLVER handle, on which a
// setup runs its independent small factorisations (slot inverses, block-Jacobi
// inverses) concurrently.  One pool per host thread, reused by every setup
// that thread runs, so the stream and handle creation is paid once.
struct Lane {
    cudaStream_t s = nullptr;
    cusolverDnHandle_t h = nullptr;
    cudaEvent_t ev = nullptr;
};
struct LanePool {
    int device = -1;
    std::vector<Lane> lanes;
    cublasHandle_t blas = nullptr;          // batched LU of the slot matrices
    void clear() {
        for (Lane& l : lanes) {
            if (l.h) cusolverDnDestroy(l.h);
            if (l.ev) cudaEventDestroy(l.ev);
            if (l.s) cudaStreamDestroy(l.s);
        }
        lanes.clear();
        if (blas) cublasDestroy(blas);
        blas = nullptr;
    }
    ~LanePool() { clear(); }
};
static thread_local LanePool t_lanes;
static constexpr int kSetupLanes = 16;

static std::vector<Lane>& setup_lanes() {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (t_lanes.device != dev) {
        t_lanes.clear();
        t_lanes.device = dev;
    }
    while ((int)t_lanes.lanes.size() < kSetupLanes) {
        Lane l;
        CK(cudaStreamCreateWithFlags(&l.s, cudaStreamNonBlocking));
        t_lanes.lanes.push_back(l);
        CK(cudaEventCreateWithFlags(&t_lanes.lanes.back().ev, cudaEventDisableTiming));
        CS(cusolverDnCreate(&t_lanes.lanes.back().h));
        CS(cusolverDnSetStream(t_lanes.lanes.back().h, l.s));
    }
    return t_lanes.lanes;
}

// Waits for every lane when a setup ends, normally or by an exception, so
// that no lane still uses the setup's temporary buffers when they are freed.
struct LaneGuard {
    std::vector<Lane>* lanes = nullptr;
    cudaEvent_t ev = nullptr;
    ~LaneGuard() {
        if (lanes)
            for (Lane& l : *lanes) cudaStreamSynchronize(l.s);
        if (ev) cudaEventDestroy(ev);
    }
};

static void setup_solver(Solver& S) {
    NvtxRange nvtx_range("smpm setup");
    auto t0 = std::chrono::steady_clock::now();
    // SMPM_TRACE_SETUP=1: per-phase wall times of the setup on stderr
    const bool trace = std::getenv("SMPM_TRACE_SETUP") != nullptr;
    if (const char* e = std::getenv("SMPM_MIRROR")) S.mirror_mode = std::atoi(e) == 0 ? 0 : 1;
    auto tp = t0;
    std::string trace_line;
    auto phase = [&](const char* name) {
        if (!trace) return;
        cudaStreamSynchronize(S.stream);
        const auto t = std::chrono::steady_clock::now();
        char buf[96];
        snprintf(buf, sizeof(buf), " %s=%.2f", name, std::chrono::duration<double, std::milli>(t - tp).count());
        trace_line += buf;
        tp = t;
    };
    Geometry& g = S.g;
    const int n = g.n, fz = g.fz, nfz = n * fz, f2 = 2 * fz, f4 = 4 * fz, mx = g.mx, ng = g.ng, d = g.d;
    cudaStream_t st = S.stream;
    CS(cusolverDnCreate(&S.sol));
    CS(cusolverDnSetStream(S.sol, st));
    S.kp = 2LL * fz * mx;
    S.ld = ((S.kp + fz + 31) / 32) * 32;
    S.restart = S.opt.restart > 0 ? S.opt.restart : 64;
    S.max_iter = S.opt.max_iter > 0 ? S.opt.max_iter : 2000;
    if (S.restart > 512) throw Err{SMPM_EINVAL, "restart above 512"};

    // strip classes and block-Jacobi block classes
    S.strip_cls.assign(mx, 1);
    S.strip_cls[0] = 0;
    S.strip_cls[mx - 1] = 2;
    const int nif = mx - 1;
    S.P = (nif + 1) / 2;
    std::vector<std::array<int, 3>> sig;
    S.pair_mc.assign(S.P, 0);
    for (int p = 0; p < S.P; ++p) {
        std::array<int, 3> sgn{S.strip_cls[2 * p], S.strip_cls[2 * p + 1], (2 * p + 1 < nif) ? S.strip_cls[2 * p + 2] : -1};
        auto it = std::find(sig.begin(), sig.end(), sgn);
        if (it == sig.end()) { sig.push_back(sgn); it = sig.end() - 1; }
        S.pair_mc[p] = (int)(it - sig.begin());
    }
    S.nmc = (int)sig.size();
    S.mc_single.resize(S.nmc);
    for (int c = 0; c < S.nmc; ++c) S.mc_single[c] = sig[c][2] < 0 ? 1 : 0;

    const int nop = S.nop;
    S.sA = (long long)nfz * nfz;
    S.sW = (long long)f2 * nfz;
    S.sG = (long long)f2 * f2;
    S.sM = (long long)f4 * f4;
    S.sRho = 3LL * 2 * ng * f2;
    S.sK = (long long)d * d;
    // 1-D factors (host)
    std::vector<double> Ax[3], beta[3], Lz;
    for (int c = 0; c < 3; ++c) {
        strip_x_operator(g, c, Ax[c]);
        face_flux_rows(g, c, beta[c]);
    }
    z_operator(g, Lz);
    phase("host_1d");
    // fast strip solver: block-diagonalise the three n x n x-factors (k-independent)
    std::vector<double> Qh[3], Qih[3], al[3], be[3];
    S.fss = true;
    // Mirror symmetry: with uniform h_x the east boundary strip's x-factor is
    // the west one's reflected (J Ax_0 J, J the order reversal) to rounding;
    // then Ax_2 = (J Q_0) B_0 (J Q_0)^-1 and class 2 shares class 0's slot
    // inverses (the refinement residual still uses the exact Ax_2).
    {
        double diff = 0.0, amax = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                amax = std::max(amax, std::fabs(Ax[0][(size_t)i * n + j]));
                diff = std::max(diff, std::fabs(Ax[0][(size_t)(n - 1 - i) * n + (n - 1 - j)] - Ax[2][(size_t)i * n + j]));
            }
        S.slot_cls[2] = (diff <= 1e-13 * amax) ? 0 : 2;
    }
    for (int c = 0; c < 3 && S.fss; ++c) {
        std::string msg;
        if (S.slot_cls[c] != c) {
            const int c0 = S.slot_cls[c];
            Qh[c].assign((size_t)n * n, 0.0);
            Qih[c].assign((size_t)n * n, 0.0);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    Qh[c][(size_t)i * n + j] = Qh[c0][(size_t)(n - 1 - i) * n + j];     // J Q_0
                    Qih[c][(size_t)i * n + j] = Qih[c0][(size_t)i * n + (n - 1 - j)];   // Q_0^-1 J
                }
            al[c] = al[c0];
            be[c] = be[c0];
            S.sl_start[c] = S.sl_start[c0];
            S.sl_size[c] = S.sl_size[c0];
            continue;
        }
        if (!real_block_diagonalise(Ax[c], n, Qh[c], Qih[c], S.sl_start[c], S.sl_size[c], al[c], be[c], msg))
            S.fss = false;
    }
    if (S.fss) {
        S.ns1 = S.ns2 = 0;
        for (int c = 0; c < 3; ++c) {
            int c1 = 0, c2 = 0;
            S.sl_idx[c].resize(S.sl_size[c].size());
            for (size_t t = 0; t < S.sl_size[c].size(); ++t) S.sl_idx[c][t] = S.sl_size[c][t] == 1 ? c1++ : c2++;
            S.ns1 = std::max(S.ns1, c1);
            S.ns2 = std::max(S.ns2, c2);
        }
        // With uniform h_z (and the same Neumann condition at the bottom and
        // the top) L_z commutes with the reversal J of the z-nodes, and so does
        // every slot matrix L_z + s I and its 2 x 2 block form.  In the basis
        // of the node pairs (p, J p) a slot matrix is [[A, B], [B, A]], so its
        // inverse is the mirror form with halves (A + B)^-1 / 2 and
        // (A - B)^-1 / 2: two inversions of half the size (a quarter of the
        // FLOPs) and slot products on half-size matrices.  The refinement step
        // of every fast solve uses the exact operator, so rounding-level
        // differences of the halves do not reach a result.
        S.zmir = false;
        if (fz % 2 == 0 && S.mirror_mode != 0) {
            double diff = 0.0, amax = 0.0;
            for (int i = 0; i < fz; ++i)
                for (int j = 0; j < fz; ++j) {
                    amax = std::max(amax, std::fabs(Lz[(size_t)i * fz + j]));
                    diff = std::max(diff, std::fabs(Lz[(size_t)(fz - 1 - i) * fz + (fz - 1 - j)] - Lz[(size_t)i * fz + j]));
                }
            S.zmir = diff <= 1e-13 * amax;
        }
        if (S.zmir) {
            const long long c1 = (long long)nop * 3 * std::max(S.ns1, 1), c2 = (long long)nop * 3 * std::max(S.ns2, 1);
            S.S1h = S.dalloc<double>((size_t)c1 * fz * fz / 2, S.allocs);
            S.S2h = S.dalloc<double>((size_t)c2 * 2 * fz * fz, S.allocs);
        } else {
            S.S1 = S.dalloc<double>((size_t)nop * 3 * std::max(S.ns1, 1) * fz * fz, S.allocs);
            S.S2 = S.dalloc<double>((size_t)nop * 3 * std::max(S.ns2, 1) * 4 * fz * fz, S.allocs);
        }
        std::vector<double> q3(3 * (size_t)n * n), qi3(3 * (size_t)n * n), b3(3 * 2 * (size_t)n);
        for (int c = 0; c < 3; ++c) {
            std::copy(Qh[c].begin(), Qh[c].end(), q3.begin() + (size_t)c * n * n);
            std::copy(Qih[c].begin(), Qih[c].end(), qi3.begin() + (size_t)c * n * n);
            std::copy(beta[c].begin(), beta[c].end(), b3.begin() + (size_t)c * 2 * n);
        }
        S.d_Q = S.dalloc<double>(q3.size(), S.allocs);
        S.d_Qinv = S.dalloc<double>(qi3.size(), S.allocs);
        S.d_beta = S.dalloc<double>(b3.size(), S.allocs);
        upload(S.d_Q, q3, st);
        upload(S.d_Qinv, qi3, st);
        upload(S.d_beta, b3, st);
        std::vector<double> ax3(3 * (size_t)n * n);
        for (int c = 0; c < 3; ++c) std::copy(Ax[c].begin(), Ax[c].end(), ax3.begin() + (size_t)c * n * n);
        S.d_Ax3 = S.dalloc<double>(ax3.size(), S.allocs);
        upload(S.d_Ax3, ax3, st);
        S.d_Lz = S.dalloc<double>(Lz.size(), S.allocs);
        upload(S.d_Lz, Lz, st);
        std::vector<int> zlo(fz, 0), zhi(fz, 0);
        for (int Z = 0; Z < fz; ++Z) {
            int lo = fz, hi = 0;
            for (int j = 0; j < fz; ++j)
                if (Lz[(size_t)Z * fz + j] != 0.0) { lo = std::min(lo, j); hi = std::max(hi, j + 1); }
            zlo[Z] = lo < hi ? lo : 0;
            zhi[Z] = hi;
        }
        S.d_zlo = S.dalloc<int>(fz, S.allocs);
        S.d_zhi = S.dalloc<int>(fz, S.allocs);
        CK(cudaMemcpyAsync(S.d_zlo, zlo.data(), fz * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(S.d_zhi, zhi.data(), fz * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        std::vector<int> c3 = {0, 1, 2};
        S.d_cls3 = S.dalloc<int>(3, S.allocs);
        CK(cudaMemcpyAsync(S.d_cls3, c3.data(), 3 * sizeof(int), cudaMemcpyHostToDevice, st));
        std::vector<int> lo1(nop * 3 * std::max(S.ns1, 1), 0), hi1(lo1.size(), fz);
        std::vector<int> lo2(nop * 3 * std::max(S.ns2, 1), 0), hi2(lo2.size(), 2 * fz);
        auto upi = [&](int*& dptr, const std::vector<int>& v) {
            dptr = S.dalloc<int>(v.size(), S.allocs);
            CK(cudaMemcpyAsync(dptr, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        };
        upi(S.rl_S1, lo1); upi(S.rh_S1, hi1); upi(S.rl_S2, lo2); upi(S.rh_S2, hi2);
        CK(cudaStreamSynchronize(st));
    } else {
        S.Ainv = S.dalloc<double>((size_t)nop * 3 * S.sA, S.allocs);
        S.W = S.dalloc<double>((size_t)nop * 3 * S.sW, S.allocs);
    }
    phase("fss_factors");
    S.G = S.dalloc<double>((size_t)nop * 3 * S.sG, S.allocs);
    S.Minv = S.dalloc<double>((size_t)nop * S.nmc * S.sM, S.allocs);
    S.rho = S.dalloc<double>((size_t)nop * S.sRho, S.allocs);
    S.K = S.dalloc<double>((size_t)nop * S.sK, S.allocs);

    // valid output rows per matrix
    {
        std::vector<int> lo(nop * 3), hi(nop * 3), loM(nop * S.nmc), hiM(nop * S.nmc), loA(nop * 3), hiA(nop * 3);
        for (int o = 0; o < nop; ++o) {
            for (int c = 0; c < 3; ++c) {
                lo[o * 3 + c] = c == 0 ? fz : 0;
                hi[o * 3 + c] = c == 2 ? fz : f2;
                loA[o * 3 + c] = 0;
                hiA[o * 3 + c] = nfz;
            }
            for (int c = 0; c < S.nmc; ++c) {
                loM[o * S.nmc + c] = 0;
                hiM[o * S.nmc + c] = S.mc_single[c] ? f2 : f4;
            }
        }
        auto up = [&](int*& dptr, const std::vector<int>& v) {
            dptr = S.dalloc<int>(v.size(), S.allocs);
            CK(cudaMemcpyAsync(dptr, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        };
        up(S.rl_GW, lo); up(S.rh_GW, hi); up(S.rl_M, loM); up(S.rh_M, hiM); up(S.rl_A, loA); up(S.rh_A, hiA);
        up(S.d_strip_cls, S.strip_cls);
        CK(cudaStreamSynchronize(st));
    }
    S.d_tau_z = S.dalloc<double>(g.mz, S.allocs);
    S.d_hz = S.dalloc<double>(g.mz, S.allocs);
    S.d_wq = S.dalloc<double>(n, S.allocs);
    upload(S.d_tau_z, g.tau_z, st);
    upload(S.d_hz, g.hz, st);
    upload(S.d_wq, g.w, st);

    std::vector<void*> tmp;
    double* dAx = S.dalloc<double>(3 * (size_t)n * n, tmp);
    double* dbeta = S.dalloc<double>(3 * 2 * (size_t)n, tmp);
    double* dLz = S.dalloc<double>((size_t)fz * fz, tmp);
    for (int c = 0; c < 3; ++c) {
        CK(cudaMemcpyAsync(dAx + (size_t)c * n * n, Ax[c].data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dbeta + (size_t)c * 2 * n, beta[c].data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice, st));
    }
    upload(dLz, Lz, st);

    // LU workspace sized for the largest matrix (the dense strip inverses of
    // the path without the fast strip solver, else the block-Jacobi blocks)
    const int mmax = S.fss ? f4 : std::max(nfz, f4);
    double *dtmp = nullptr, *dwork = nullptr;
    int *dipiv = nullptr, *dinfo = nullptr;
    int lwork = 0;
    CS(cusolverDnDgetrf_bufferSize(S.sol, mmax, mmax, nullptr, mmax, &lwork));
    if (!S.fss) {
        dtmp = S.dalloc<double>((size_t)mmax * mmax, tmp);
        dwork = S.dalloc<double>((size_t)std::max(lwork, 1), tmp);
        dipiv = S.dalloc<int>((size_t)mmax, tmp);
        dinfo = S.dalloc<int>(1, tmp);
    }

    phase("alloc_upload");
    // null vectors (k^2 = 0): u_L = u_Lx (x) u_Lz, u_S = E^T u_L / ||E^T u_L||
    std::vector<double> uS_h;
    for (int o = 0; o < nop; ++o)
        if (S.k2[o] == 0.0) S.singular_op = o;
    if (S.singular_op >= 0) {
        std::vector<double> ux, uz;
        std::string msg;
        if (!left_null_x(g, ux, msg) || !left_null_z(g, uz, msg)) throw Err{SMPM_EBREAKDOWN, msg};
        std::vector<double> uL_h((size_t)g.r);
        for (int X = 0; X < g.nx; ++X)
            for (int Z = 0; Z < fz; ++Z) uL_h[(size_t)X * fz + Z] = ux[X] * uz[Z];
        uS_h.assign((size_t)S.ld, 0.0);
        double nrm = 0.0;
        for (int i = 0; i < mx; ++i)
            for (int sd = 0; sd < 2; ++sd) {
                const int F = 2 * i + sd;
                if (F == 0 || F == 2 * mx - 1) continue;
                const int X = i * n + (sd == 0 ? 0 : g.N);
                for (int Z = 0; Z < fz; ++Z) {
                    const double v = ux[X] * uz[Z];
                    uS_h[(size_t)F * fz + Z] = v;
                    nrm += v * v;
                }
            }
        nrm = std::sqrt(nrm);
        for (double& v : uS_h) v /= nrm;
        S.uL = S.dalloc<double>((size_t)g.r, S.allocs);
        S.uS = S.dalloc<double>((size_t)S.ld, S.allocs);
        {   // S 1 = 0 (constants are in the null space of the Neumann operator)
            std::vector<double> one_h((size_t)S.ld, 0.0);
            const double v = 1.0 / std::sqrt((double)g.k);
            for (long long i = fz; i < S.kp - fz; ++i) one_h[(size_t)i] = v;
            S.oneS = S.dalloc<double>((size_t)S.ld, S.allocs);
            upload(S.oneS, one_h, st);
            CK(cudaStreamSynchronize(st));
        }
        upload(S.uL, uL_h, st);
        upload(S.uS, uS_h, st);
        CK(cudaStreamSynchronize(st));
    }

    phase("null_vectors");

    // Independent factorisations run on the setup lanes; every getrf/getrs
    // writes its own status word, checked once after the last join.
    std::vector<Lane>& lanes = setup_lanes();
    LaneGuard guard;
    guard.lanes = &lanes;
    const int L = (int)lanes.size();
    const int mlane = std::max(f4, S.fss ? f2 : 0);
    // precision 2 uses only FP32 block-Jacobi inverses: they are factorised
    // and inverted in FP32 (cuSOLVER S-getrf/getrs) from the FP64 blocks
    const bool m_fp32 = S.precision == 2;
    int lwork_f = 0;
    if (m_fp32) CS(cusolverDnSgetrf_bufferSize(S.sol, f4, f4, nullptr, f4, &lwork_f));
    struct LaneBuf { double *a, *b, *work; int* ipiv; float *af, *cf, *workf; };
    std::vector<LaneBuf> lb(L);
    for (int l = 0; l < L; ++l) {
        lb[l].a = S.dalloc<double>((size_t)mlane * mlane, tmp);
        lb[l].b = S.dalloc<double>((size_t)f2 * f2, tmp);
        lb[l].work = S.dalloc<double>((size_t)std::max(lwork, 1), tmp);
        lb[l].ipiv = S.dalloc<int>((size_t)mlane, tmp);
        lb[l].af = lb[l].cf = lb[l].workf = nullptr;
        if (m_fp32) {
            lb[l].af = S.dalloc<float>((size_t)f4 * f4, tmp);
            lb[l].cf = S.dalloc<float>((size_t)f4 * f4, tmp);
            lb[l].workf = S.dalloc<float>((size_t)std::max(lwork_f, 1), tmp);
        }
    }
    int n_inv = 0;
    for (int c = 0; c < 3 && S.fss; ++c) n_inv += (S.zmir ? 2 : 1) * (int)S.sl_size[c].size();
    n_inv = nop * (n_inv + S.nmc + 1);
    int* d_infos = S.dalloc<int>((size_t)2 * n_inv, tmp);
    CK(cudaMemsetAsync(d_infos, 0, sizeof(int) * 2 * n_inv, st));
    int inv_used = 0, next_lane = 0;
    cudaEvent_t fork_ev = nullptr;
    CK(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
    guard.ev = fork_ev;
    auto fork = [&] {
        CK(cudaEventRecord(fork_ev, st));
        for (Lane& ln : lanes) CK(cudaStreamWaitEvent(ln.s, fork_ev, 0));
        next_lane = 0;
    };
    auto join = [&] {
        for (Lane& ln : lanes) {
            CK(cudaEventRecord(ln.ev, ln.s));
            CK(cudaStreamWaitEvent(st, ln.ev, 0));
        }
    };
    // dst <- src^-1 on lane l (row-major; src destroyed)
    auto invert_on = [&](int l, double* src, double* dst, int m) {
        if (inv_used >= n_inv) throw Err{SMPM_ECUDA, "setup: inversion count exceeded"};
        int* info = d_infos + 2 * inv_used++;
        k_identity(dst, m, lanes[l].s);
        CS(cusolverDnDgetrf(lanes[l].h, m, m, src, m, lb[l].work, lb[l].ipiv, info));
        CS(cusolverDnDgetrs(lanes[l].h, CUBLAS_OP_N, m, m, src, m, lb[l].ipiv, dst, m, info + 1));
    };

    // destination of slot t of class c, operator o: the full inverse, or its
    // two mirror halves (first (A + B)^-1 / 2, then (A - B)^-1 / 2)
    auto slot_dst = [&](int o, int c, size_t t) -> double* {
        const int sz = S.sl_size[c][t], idx = S.sl_idx[c][t];
        if (S.zmir)
            return sz == 1 ? S.S1h + (((size_t)o * 3 + c) * std::max(S.ns1, 1) + idx) * fz * fz / 2
                           : S.S2h + (((size_t)o * 3 + c) * std::max(S.ns2, 1) + idx) * 2 * fz * fz;
        return sz == 1 ? S.S1 + (((size_t)o * 3 + c) * std::max(S.ns1, 1) + idx) * fz * fz
                       : S.S2 + (((size_t)o * 3 + c) * std::max(S.ns2, 1) + idx) * 4 * fz * fz;
    };
    // phase 1: slot inverses of B_c (+) L_z - k^2 for every operator (Sec. 5:
    // only the shift depends on k).  Slot matrices up to kBatchedMax rows go
    // through one batched LU and inversion per size (cuBLAS getrf/getriBatched,
    // on the solver's stream); larger ones through cuSOLVER on the lanes
    // (measured: batched 0.21 vs 0.66 ms for the 14-row slots of 64x2 order 6,
    // 94 vs 19 ms for the 272-row slots of 1024x16 order 16).
    constexpr int kBatchedMax = 128;
    constexpr int kGjMinGlobal = 32;     // Gauss-Jordan in global memory only for this many matrices or more
    if (S.fss) {
        if (!t_lanes.blas) {
            if (cublasCreate(&t_lanes.blas) != CUBLAS_STATUS_SUCCESS) throw Err{SMPM_ECUDA, "cublasCreate failed"};
        }
        cublasSetStream(t_lanes.blas, st);
        for (int sz = 1; sz <= 2; ++sz) {
            const int m = sz * fz;
            if (m > kBatchedMax || S.zmir) continue;
            std::vector<double*> src_p, dst_p;
            std::vector<std::array<int, 3>> items;
            for (int o = 0; o < nop; ++o)
                for (int c = 0; c < 3; ++c) {
                    if (S.slot_cls[c] != c) continue;
                    for (size_t t = 0; t < S.sl_size[c].size(); ++t)
                        if (S.sl_size[c][t] == sz) items.push_back({o, c, (int)t});
                }
            const int nb = (int)items.size();
            if (nb == 0) continue;
            double* work = S.dalloc<double>((size_t)nb * m * m, tmp);
            for (int i = 0; i < nb; ++i) {
                const int o = items[i][0], c = items[i][1], t = items[i][2];
                double* a = work + (size_t)i * m * m;
                k_build_slot(a, dLz, fz, sz, al[c][t] - S.k2[o], be[c][t], st);
                src_p.push_back(a);
                dst_p.push_back(slot_dst(o, c, t));
            }
            double** d_src = S.dalloc<double*>((size_t)nb, tmp);
            double** d_dst = S.dalloc<double*>((size_t)nb, tmp);
            int* piv = S.dalloc<int>((size_t)nb * m, tmp);
            int* inf = S.dalloc<int>((size_t)2 * nb, tmp);
            CK(cudaMemcpyAsync(d_src, src_p.data(), nb * sizeof(double*), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(d_dst, dst_p.data(), nb * sizeof(double*), cudaMemcpyHostToDevice, st));
            // row-major buffers read as their transposes: inv(A^T) = inv(A)^T, i.e.
            // the row-major inverse, is what getriBatched writes
            if (cublasDgetrfBatched(t_lanes.blas, m, d_src, m, piv, inf, nb) != CUBLAS_STATUS_SUCCESS ||
                cublasDgetriBatched(t_lanes.blas, m, (const double* const*)d_src, m, piv, d_dst, m, inf + nb, nb) !=
                    CUBLAS_STATUS_SUCCESS)
                throw Err{SMPM_ECUDA, "batched slot inversion failed"};
            std::vector<int> h_inf((size_t)2 * nb);
            CK(cudaMemcpyAsync(h_inf.data(), inf, h_inf.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (int v : h_inf)
                if (v != 0) throw Err{SMPM_EBREAKDOWN, "singular slot matrix (batched getrf info " + std::to_string(v) + ")"};
        }
    }
    if (S.fss && !S.zmir) {
        fork();
        for (int o = 0; o < nop; ++o)
            for (int c = 0; c < 3; ++c) {
                if (S.slot_cls[c] != c) continue;          // shares another class's slots
                for (size_t t = 0; t < S.sl_size[c].size(); ++t) {
                    const int sz = S.sl_size[c][t], m = sz * fz;
                    if (m <= kBatchedMax) continue;       // done by the batched inversion
                    const int l = next_lane++ % L;
                    k_build_slot(lb[l].a, dLz, fz, sz, al[c][t] - S.k2[o], be[c][t], lanes[l].s);
                    invert_on(l, lb[l].a, slot_dst(o, c, t), m);
                }
            }
        join();
    }
    if (S.fss && S.zmir) {
        // mirror halves: every half of every slot and operator of one size
        // inverted by one Gauss-Jordan launch (one CTA per matrix): the
        // per-matrix cuSOLVER calls spent ~3 ms each in launch latency on
        // matrices of 136-272 rows, two orders of magnitude above their FLOPs
        for (int sz = 1; sz <= 2; ++sz) {
            const int h = sz * fz / 2;
            std::vector<const double*> src_p;
            std::vector<double*> dst_p;
            std::vector<std::array<int, 3>> items;
            for (int o = 0; o < nop; ++o)
                for (int c = 0; c < 3; ++c) {
                    if (S.slot_cls[c] != c) continue;
                    for (size_t t = 0; t < S.sl_size[c].size(); ++t)
                        if (S.sl_size[c][t] == sz) items.push_back({o, c, (int)t});
                }
            const int nb = 2 * (int)items.size();
            if (nb == 0) continue;
            if (h > gj_smem_max() && nb < kGjMinGlobal) {
                // few large halves (a single operator's 2 x 2 slots): one CTA
                // per matrix would leave most SMs idle for ~5 ms, so they go
                // to cuSOLVER on the lanes, concurrently
                fork();
                for (const auto& it : items) {
                    const int o = it[0], c = it[1], t = it[2];
                    const int l = next_lane++ % L;
                    double* d = slot_dst(o, c, t);
                    k_build_slot_halves(lb[l].a, dLz, fz, sz, al[c][t] - S.k2[o], be[c][t], lanes[l].s);
                    invert_on(l, lb[l].a, d, h);
                    invert_on(l, lb[l].a + (size_t)h * h, d + (size_t)h * h, h);
                }
                join();
                continue;
            }
            double* work = S.dalloc<double>((size_t)nb * h * h, tmp);
            for (size_t it = 0; it < items.size(); ++it) {
                const int o = items[it][0], c = items[it][1], t = items[it][2];
                double* a = work + (size_t)2 * it * h * h;
                double* d = slot_dst(o, c, t);
                k_build_slot_halves(a, dLz, fz, sz, al[c][t] - S.k2[o], be[c][t], st);
                src_p.push_back(a);
                src_p.push_back(a + (size_t)h * h);
                dst_p.push_back(d);
                dst_p.push_back(d + (size_t)h * h);
            }
            const double** d_src = S.dalloc<const double*>((size_t)nb, tmp);
            double** d_dst = S.dalloc<double*>((size_t)nb, tmp);
            int* inf = S.dalloc<int>((size_t)nb, tmp);
            CK(cudaMemcpyAsync(d_src, src_p.data(), nb * sizeof(double*), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(d_dst, dst_p.data(), nb * sizeof(double*), cudaMemcpyHostToDevice, st));
            k_gj_inverse(d_src, d_dst, h, nb, inf, st);
            CK(cudaGetLastError());
            std::vector<int> h_inf((size_t)nb);
            CK(cudaMemcpyAsync(h_inf.data(), inf, h_inf.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (int v : h_inf)
                if (v != 0) throw Err{SMPM_EBREAKDOWN, "singular slot matrix half (Gauss-Jordan pivot " + std::to_string(v) + ")"};
        }
    }
    if (S.fss) phase("slot_inverses");

    // phase 2: G_c = B A_c^-1 E_c and the coarse row sums, per operator
    double *U = nullptr, *Y = nullptr, *T1 = nullptr, *T2 = nullptr;
    // fast solves of the 2 fz unit face vectors of one strip, for up to
    // kGOps operators in one refined solve per class
    constexpr int kGOps = 8;
    const int gops = std::min(nop, kGOps);
    if (S.fss) {
        U = S.dalloc<double>((size_t)gops * f2 * nfz, tmp);
        Y = S.dalloc<double>((size_t)gops * f2 * nfz, tmp);
        T1 = S.dalloc<double>((size_t)gops * f2 * nfz, tmp);
        T2 = S.dalloc<double>((size_t)gops * f2 * nfz, tmp);
        for (int q = 0; q < gops; ++q) k_unit_faces(U + (size_t)q * f2 * nfz, n, fz, st);
        for (int o0 = 0; o0 < nop; o0 += gops) {
            const int no = std::min(gops, nop - o0);
            // the east boundary class of a mirror-symmetric grid is the west
            // one with its two faces swapped (after both are built)
            for (int c = 0; c < 3; ++c) {
                if (c == 1 && mx < 3) {
                    for (int o = o0; o < o0 + no; ++o) k_fill(S.G + ((size_t)o * 3 + c) * S.sG, S.sG, 0.0, st);
                    continue;
                }
                if (S.slot_cls[c] != c) continue;
                fss_setup(S, o0, no, c, f2, U, Y, T1, T2, tmp);
                for (int q = 0; q < no; ++q)
                    k_g_from_solves(S.G + ((size_t)(o0 + q) * 3 + c) * S.sG, Y + (size_t)q * f2 * nfz,
                                    S.d_beta + (size_t)c * 2 * n, n, fz, c, st);
            }
            for (int o = o0; o < o0 + no; ++o)
                for (int c = 0; c < 3; ++c)
                    if (S.slot_cls[c] != c && !(c == 1 && mx < 3)) {
                        double* G = S.G + (size_t)o * 3 * S.sG;
                        k_mirror_blocks(G + c * S.sG, G + S.slot_cls[c] * S.sG, fz, 2, st);
                    }
        }
    }
    for (int o = 0; o < nop && !S.fss; ++o) {
        const double k2 = S.k2[o];
        double* G = S.G + (size_t)o * 3 * S.sG;
        for (int c = 0; c < 3; ++c) {
            double* Ainv = S.Ainv + (size_t)o * 3 * S.sA;
            double* W = S.W + (size_t)o * 3 * S.sW;
            if (c == 1 && mx < 3) {  // no interior strips
                k_fill(Ainv + c * S.sA, S.sA, 0.0, st);
                k_fill(W + c * S.sW, S.sW, 0.0, st);
                k_fill(G + c * S.sG, S.sG, 0.0, st);
                continue;
            }
            k_build_strip_op(dtmp, dAx + (size_t)c * n * n, dLz, k2, n, fz, st);
            invert_dense(S, dtmp, Ainv + c * S.sA, nfz, dwork, lwork, dipiv, dinfo);
            k_build_W(W + c * S.sW, Ainv + c * S.sA, dbeta + (size_t)c * 2 * n, n, fz, st);
            k_build_G(G + c * S.sG, W + c * S.sW, n, fz, c, st);
        }
    }
    // Interior strips of a uniform-h_x grid are symmetric under the reflection
    // of x about the strip centre, so G_1 = J G_1 J (J: the two faces swapped)
    // up to the rounding of its solves.  Where the computed G_1 has that
    // symmetry to 1e-11 relative (every operator), it is made exactly
    // symmetric and the Schur product of the interior strips runs in the
    // mirror form (half the FLOPs, kernels.cu); the boundary strips keep the
    // full product.  The coarse row sums and the block-Jacobi pairs are built
    // from the symmetric G_1, so every part of the method uses one operator.
    S.mirG = S.mirM = false;
    if (mx >= 3 && S.mirror_mode != 0) {
        double* dres = S.dalloc<double>((size_t)2 * nop, tmp);
        for (int o = 0; o < nop; ++o) k_mirror_asym(S.G + ((size_t)o * 3 + 1) * S.sG, fz, 2, dres + 2 * o, st);
        std::vector<double> res((size_t)2 * nop);
        CK(cudaMemcpyAsync(res.data(), dres, sizeof(double) * res.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        bool ok = true;
        for (int o = 0; o < nop; ++o) ok = ok && res[2 * o] <= 1e-11 * res[2 * o + 1];
        if (trace)
            for (int o = 0; o < nop; ++o)
                fprintf(stderr, "smpm setup: interior Schur block mirror asymmetry %.2e (op %d)\n",
                        res[2 * o] / std::max(res[2 * o + 1], 1e-300), o);
        if (ok) {
            S.mirG = true;
            const long long sh = (long long)fz * fz;
            S.Gh = S.dalloc<double>((size_t)nop * 2 * sh, S.allocs);
            for (int o = 0; o < nop; ++o) {
                double* G1 = S.G + ((size_t)o * 3 + 1) * S.sG;
                k_mirror_symmetrize(G1, fz, 2, st);
                k_mirror_halves(S.Gh + (size_t)o * 2 * sh, G1, fz, 2, st);
            }
        }
    }
    for (int o = 0; o < nop; ++o)
        for (int c = 0; c < 3; ++c)
            k_build_rho(S.rho + (size_t)o * S.sRho + (size_t)c * 2 * ng * f2, S.G + ((size_t)o * 3 + c) * S.sG, fz, ng,
                        st);
    phase("G");

    // phase 3: block-Jacobi pair blocks and their inverses (Sec. 3.2).  On a
    // mirror-symmetric grid the last pair (strips of classes 1, 1, 2) is the
    // mirror image of the first (0, 1, 1): its inverse is the first one's
    // with the four face blocks reversed.
    int mc_first = -1, mc_last = -1;
    for (int mc = 0; mc < S.nmc; ++mc) {
        if (sig[mc] == std::array<int, 3>{0, 1, 1}) mc_first = mc;
        if (sig[mc] == std::array<int, 3>{1, 1, 2}) mc_last = mc;
    }
    const bool mirror_m = S.slot_cls[2] == 0 && mc_first >= 0 && mc_last >= 0 && !m_fp32;
    if (m_fp32) {   // the FP32 inverses go straight into Minv32
        S.Minv32 = S.dalloc<float>((size_t)nop * S.nmc * S.sM, S.allocs);
    }
    fork();
    for (int o = 0; o < nop; ++o) {
        const double* G = S.G + (size_t)o * 3 * S.sG;
        for (int mc = 0; mc < S.nmc; ++mc) {
            if (mirror_m && mc == mc_last) continue;   // after the join
            const int l = next_lane++ % L;
            cudaStream_t ls = lanes[l].s;
            const double* gA = G + sig[mc][0] * S.sG;
            const double* gB = G + sig[mc][1] * S.sG;
            const double* gC = sig[mc][2] >= 0 ? G + sig[mc][2] * S.sG : nullptr;
            const int m = gC ? f4 : f2;
            double* dst = S.Minv + ((size_t)o * S.nmc + mc) * S.sM;
            if (m_fp32) {
                float* dst32 = S.Minv32 + ((size_t)o * S.nmc + mc) * S.sM;
                if (S.P == 1 && S.k2[o] == 0.0) {
                    k_identity_f(lb[l].cf, m, ls);
                } else {
                    k_build_M(lb[l].a, gA, gB, gC, fz, ls);
                    k_to_fp32(lb[l].af, lb[l].a, (long long)m * m, ls);
                    const int slot = inv_used++;
                    if (slot >= n_inv) throw Err{SMPM_ECUDA, "setup: inversion count exceeded"};
                    int* info = d_infos + 2 * slot;
                    k_identity_f(lb[l].cf, m, ls);
                    CS(cusolverDnSgetrf(lanes[l].h, m, m, lb[l].af, m, lb[l].workf, lb[l].ipiv, info));
                    CS(cusolverDnSgetrs(lanes[l].h, CUBLAS_OP_N, m, m, lb[l].af, m, lb[l].ipiv, lb[l].cf, m, info + 1));
                }
                k_pad_block_f(dst32, lb[l].cf, m, f4, ls);
                continue;
            }
            if (S.P == 1 && S.k2[o] == 0.0) {
                // m_x <= 3: the one block is all of the singular S; use M = I
                k_identity(lb[l].a, m, ls);
                k_pad_block(dst, lb[l].a, m, f4, ls);
                continue;
            }
            k_build_M(lb[l].a, gA, gB, gC, fz, ls);
            if (m == f4) {
                invert_on(l, lb[l].a, dst, m);
            } else {
                invert_on(l, lb[l].a, lb[l].b, m);
                k_pad_block(dst, lb[l].b, m, f4, ls);
            }
        }
    }
    join();
    if (mirror_m)
        for (int o = 0; o < nop; ++o)
            k_mirror_blocks(S.Minv + ((size_t)o * S.nmc + mc_last) * S.sM, S.Minv + ((size_t)o * S.nmc + mc_first) * S.sM,
                            fz, 4, st);
    // The interior pairs (strip classes 1, 1, 1) are built from the symmetric
    // G_1, so their block is symmetric under the reversal of its four faces,
    // and so is its inverse up to rounding: symmetrised, it runs in the
    // mirror form too (FP32 copies for the mixed forms below).
    S.mc_int = -1;
    for (int mc = 0; mc < S.nmc; ++mc)
        if (sig[mc] == std::array<int, 3>{1, 1, 1}) S.mc_int = mc;
    if (S.mirG && S.mc_int >= 0 && !(S.P == 1)) {
        const long long sh = 4LL * fz * fz;
        if (m_fp32) {
            S.Mh32 = S.dalloc<float>((size_t)nop * 2 * sh, S.allocs);
            for (int o = 0; o < nop; ++o)
                k_mirror_halves_f(S.Mh32 + (size_t)o * 2 * sh, S.Minv32 + ((size_t)o * S.nmc + S.mc_int) * S.sM, fz, 4,
                                  st);
        } else {
            S.Mh = S.dalloc<double>((size_t)nop * 2 * sh, S.allocs);
            for (int o = 0; o < nop; ++o) {
                double* Mi = S.Minv + ((size_t)o * S.nmc + S.mc_int) * S.sM;
                k_mirror_symmetrize(Mi, fz, 4, st);
                k_mirror_halves(S.Mh + (size_t)o * 2 * sh, Mi, fz, 4, st);
            }
        }
        S.mirM = true;
    }
    phase("M_inverses");

    // phase 4: coarse matrix C = Z^T S Z from the row sums (host), then its
    // division K on the GPU (Sec. 3.3)
    std::vector<double> rho_h((size_t)nop * S.sRho);
    CK(cudaMemcpyAsync(rho_h.data(), S.rho, sizeof(double) * rho_h.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int gs = fz / ng;
    // One deflation vector per interface (ng = 1): C is tridiagonal (an
    // interface couples to its two neighbours through the strips between
    // them), and for k^2 > 0 it is nonsingular, so K = C^-1 comes from a
    // pivoted tridiagonal LU on the host (O(d)) and one GPU thread per column
    // (O(d^2) in all) instead of a dense d x d factorisation and d solves.
    // SMPM_COARSE_DENSE=1 takes the dense path for every operator.
    const bool tri_path = ng == 1 && std::getenv("SMPM_COARSE_DENSE") == nullptr;
    bool any_dense = false;
    for (int o = 0; o < nop; ++o) any_dense |= !(tri_path && S.k2[o] > 0.0);
    int lwork_d = 0;
    double *dC = nullptr, *dwork_d = nullptr, *duC = nullptr, *dw = nullptr;
    int* dipiv_d = nullptr;
    std::vector<double> C, uC;
    if (any_dense) {
        CS(cusolverDnDgetrf_bufferSize(S.sol, d, d, S.K, d, &lwork_d));
        dC = S.dalloc<double>((size_t)d * d, tmp);
        dwork_d = S.dalloc<double>((size_t)std::max(lwork_d, 1), tmp);
        dipiv_d = S.dalloc<int>((size_t)d, tmp);
        duC = S.dalloc<double>((size_t)d, tmp);
        dw = S.dalloc<double>((size_t)d, tmp);
        C.resize((size_t)d * d);
    }
    double* dfac = S.dalloc<double>((size_t)nop * 4 * std::max(d, 1), tmp);
    int* dswap = S.dalloc<int>((size_t)nop * std::max(d, 1), tmp);
    std::vector<std::vector<double>> tri_fac(nop);       // kept until the copies have run
    std::vector<std::vector<int>> tri_swap(nop);
    for (int o = 0; o < nop; ++o) {
        const double k2 = S.k2[o];
        const double* rho_o = rho_h.data() + (size_t)o * S.sRho;
        // gsum[cls][side][g][half][g'] = sum over group g' of half `half` of rho[cls][side][g]
        auto rh = [&](int cls, int side, int gg) { return rho_o + ((size_t)(cls * 2 + side) * ng + gg) * f2; };
        auto gsum = [&](int cls, int side, int gg, int half, int gp) {
            const double* v = rh(cls, side, gg) + half * fz + gp * gs;
            double sm = 0.0;
            for (int z = 0; z < gs; ++z) sm += v[z];
            return sm;
        };
        if (tri_path && k2 > 0.0) {
            // C(t, t), C(t+1, t), C(t-1, t) as in the dense assembly below
            std::vector<double> dl((size_t)std::max(d - 1, 0)), dd((size_t)d), du((size_t)std::max(d - 1, 0)), du2;
            double sums[3][2][2];                        // gsum(cls, side, 0, half, 0): 12 values per operator
            for (int cl = 0; cl < 3; ++cl)
                for (int side = 0; side < 2; ++side)
                    for (int half = 0; half < 2; ++half) sums[cl][side][half] = gsum(cl, side, 0, half, 0);
            for (int t = 0; t < nif; ++t) {
                const int cl_r = S.strip_cls[t + 1], cl_l = S.strip_cls[t];
                dd[t] = 2.0 * gs + sums[cl_r][0][0] + sums[cl_l][1][1];
                if (t >= 1) du[t - 1] = sums[cl_l][1][0];
                if (t + 1 <= nif - 1) dl[t] = sums[cl_r][0][1];
            }
            std::vector<int>& sw = tri_swap[o];
            if (!tridiag_lu(d, dl, dd, du, du2, sw))
                throw Err{SMPM_EBREAKDOWN, "singular coarse matrix (zero pivot of the tridiagonal LU)"};
            std::vector<double>& fac = tri_fac[o];
            fac.reserve((size_t)4 * d);
            fac.insert(fac.end(), dl.begin(), dl.end());
            fac.insert(fac.end(), dd.begin(), dd.end());
            fac.insert(fac.end(), du.begin(), du.end());
            fac.insert(fac.end(), du2.begin(), du2.end());
            double* fo = dfac + (size_t)o * 4 * std::max(d, 1);
            int* so = dswap + (size_t)o * std::max(d, 1);
            CK(cudaMemcpyAsync(fo, fac.data(), sizeof(double) * fac.size(), cudaMemcpyHostToDevice, st));
            if (!sw.empty()) CK(cudaMemcpyAsync(so, sw.data(), sizeof(int) * sw.size(), cudaMemcpyHostToDevice, st));
            k_tridiag_inverse(S.K + (size_t)o * S.sK, fo, so, d, st);
            continue;
        }
        std::fill(C.begin(), C.end(), 0.0);
        for (int t = 0; t < nif; ++t)
            for (int gg = 0; gg < ng; ++gg) {
                const int col = t * ng + gg;
                const int cl_r = S.strip_cls[t + 1], cl_l = S.strip_cls[t];
                C[(size_t)col * d + col] += 2.0 * gs;
                for (int gp = 0; gp < ng; ++gp) {
                    C[(size_t)(t * ng + gp) * d + col] += gsum(cl_r, 0, gg, 0, gp) + gsum(cl_l, 1, gg, 1, gp);
                    if (t >= 1) C[(size_t)((t - 1) * ng + gp) * d + col] += gsum(cl_l, 1, gg, 0, gp);
                    if (t + 1 <= nif - 1) C[(size_t)((t + 1) * ng + gp) * d + col] += gsum(cl_r, 0, gg, 1, gp);
                }
            }
        const double* uCp = nullptr;
        if (k2 == 0.0) {  // u_C = Z^T u_S normalised (Sec. 3.3)
            uC.assign(d, 0.0);
            double nrm = 0.0;
            for (int t = 0; t < nif; ++t)
                for (int gg = 0; gg < ng; ++gg) {
                    double sm = 0.0;
                    for (int z = 0; z < gs; ++z)
                        sm += uS_h[(size_t)(2 * t + 1) * fz + gg * gs + z] + uS_h[(size_t)(2 * t + 2) * fz + gg * gs + z];
                    uC[t * ng + gg] = sm;
                    nrm += sm * sm;
                }
            nrm = std::sqrt(nrm);
            for (double& v : uC) v /= nrm;
            uCp = uC.data();
        }
        coarse_matrix(C, d, fz / ng, uCp);   // C + alpha u_C 1^T / sqrt(d) when singular
        double* K = S.K + (size_t)o * S.sK;
        upload(dC, C, st);
        if (inv_used >= n_inv) throw Err{SMPM_ECUDA, "setup: inversion count exceeded"};
        int* info = d_infos + 2 * inv_used++;
        k_identity(K, d, st);
        CS(cusolverDnDgetrf(S.sol, d, d, dC, d, dwork_d, dipiv_d, info));
        CS(cusolverDnDgetrs(S.sol, CUBLAS_OP_N, d, d, dC, d, dipiv_d, K, d, info + 1));
        if (uCp) {
            upload(duC, uC, st);
            k_project_coarse(K, dw, duC, d, st);
        }
        CK(cudaStreamSynchronize(st));   // C and uC are reused by the next operator
    }
    std::vector<int> infos((size_t)2 * inv_used);
    if (inv_used > 0) {
        CK(cudaMemcpyAsync(infos.data(), d_infos, sizeof(int) * infos.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    for (int v : infos)
        if (v != 0) throw Err{SMPM_EBREAKDOWN, "singular strip slot, block-Jacobi or coarse matrix (getrf info " + std::to_string(v) + ")"};
    phase("coarse");
    if (S.precision == 1) {
        S.Minv32 = S.dalloc<float>((size_t)nop * S.nmc * S.sM, S.allocs);
        k_to_fp32(S.Minv32, S.Minv, (long long)nop * S.nmc * S.sM, st);
        if (S.mirM) {
            S.Mh32 = S.dalloc<float>((size_t)nop * 2 * 4 * fz * fz, S.allocs);
            k_to_fp32(S.Mh32, S.Mh, (long long)nop * 2 * 4 * fz * fz, st);
        }
        // An FP32 copy of an ill-conditioned block inverse (large k^2 on fine
        // grids) turns the preconditioner into noise: measure the FP32 apply's
        // relative error on a sign vector for every block, and keep the FP64
        // blocks for precision 1 when it exceeds 1e-3.
        double* q = S.dalloc<double>((size_t)nop * S.nmc, tmp);
        k_fp32_quality(S.Minv, S.Minv32, f4, S.sM, nop * S.nmc, q, st);
        std::vector<double> qh((size_t)nop * S.nmc);
        CK(cudaMemcpyAsync(qh.data(), q, sizeof(double) * qh.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        S.fp32_err = 0.0;
        for (double v : qh) S.fp32_err = std::max(S.fp32_err, v);
        S.bj32_ok = S.fp32_err <= 1e-3;
        if (trace) fprintf(stderr, "smpm setup: FP32 block-Jacobi relative apply error %.2e\n", S.fp32_err);
    }
    if (S.precision == 2) {
        S.G32 = S.dalloc<float>((size_t)nop * 3 * S.sG, S.allocs);
        k_to_fp32(S.G32, S.G, (long long)nop * 3 * S.sG, st);
        if (S.mirG) {
            S.Gh32 = S.dalloc<float>((size_t)nop * 2 * fz * fz, S.allocs);
            k_to_fp32(S.Gh32, S.Gh, (long long)nop * 2 * fz * fz, st);
        }
    }
    // SMPM_OZAKI (bit mask): 1 = the FP64 Schur and block-Jacobi products on
    // the tensor cores at FP64 accuracy (56-bit digit splits); 2 = the FP32
    // products (the FP32 block-Jacobi of precision 1, the inner Schur and
    // block-Jacobi products of precision 2) on the tensor cores at the 24-bit
    // accuracy of FP32 (4-5 digits).  Their class matrices are split into BF16
    // digit tensors here, keyed by the matrix array the products name.
    if (const char* oe = std::getenv("SMPM_OZAKI")) S.oz_mask = std::atoi(oe) & 3;
    if (S.precision == 0) S.oz_mask &= 1;
    S.oz = S.oz_mask != 0;
    if (S.oz) {
        auto split = [&](const void* key, const double* mats, const float* mats_f, long long stride, int nmat, int Mm,
                         int bits) {
            Solver::OzMat z;
            if (!oz_choose(Mm, z.S, z.beta, z.N, bits)) return;
            z.mt_n = (Mm + 127) / 128;
            z.kcn = (Mm + 127) / 128;
            z.dig_stride = (long long)z.mt_n * z.kcn * z.S * 128 * 128;
            z.rexp_stride = (long long)z.mt_n * 128;
            z.dig = S.dalloc<unsigned short>((size_t)nmat * z.dig_stride, S.allocs);
            z.rexp = S.dalloc<int>((size_t)nmat * z.rexp_stride, S.allocs);
            if (mats)
                k_oz_split_rows(mats, stride, nmat, Mm, Mm, z.S, z.beta, z.mt_n, z.kcn, z.dig, z.dig_stride, z.rexp,
                                z.rexp_stride, st);
            else
                k_oz_split_rows_f(mats_f, stride, nmat, Mm, Mm, z.S, z.beta, z.mt_n, z.kcn, z.dig, z.dig_stride,
                                  z.rexp, z.rexp_stride, st);
            S.ozmats[reinterpret_cast<const double*>(key)] = z;
        };
        // precision 2 keeps its block-Jacobi inverses in FP32 only
        const bool minv64 = S.precision != 2;
        if (S.oz_mask & 1) {
            split(S.G, S.G, nullptr, S.sG, nop * 3, 2 * fz, 56);
            if (minv64) split(S.Minv, S.Minv, nullptr, S.sM, nop * S.nmc, 4 * fz, 56);
        }
        if (S.oz_mask & 2) {
            // digits of the FP64 matrix where the handle keeps one (more
            // accurate than its FP32 copy), of the FP32 copy otherwise
            if (S.G32) split(S.G32, S.G, nullptr, S.sG, nop * 3, 2 * fz, 24);
            if (S.Minv32) {
                if (minv64) split(S.Minv32, S.Minv, nullptr, S.sM, nop * S.nmc, 4 * fz, 24);
                else split(S.Minv32, nullptr, S.Minv32, S.sM, nop * S.nmc, 4 * fz, 24);
            }
        }
        S.d_ozerr = S.dalloc<int>(1, S.allocs);
        CK(cudaMemsetAsync(S.d_ozerr, 0, sizeof(int), st));
    }
    CK(cudaStreamSynchronize(st));
    S.free_list(tmp);
    S.setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (trace)
        fprintf(stderr, "smpm setup %dx%d p%d nop=%d fss=%d zmir=%d slots(1x1, 2x2 per class)=%d,%d total=%.2f:%s\n",
                g.mx, g.mz, g.N, S.nop, (int)S.fss, (int)S.zmir, S.ns1, S.ns2,
                S.setup_ms, trace_line.c_str());
}

// ---------------------------------------------------------------------------
// Workspace and tiles
// ---------------------------------------------------------------------------

static void ensure_workspace(Solver& S, int R) {
    if (R <= S.Rcap) return;
    CK(cudaStreamSynchronize(S.stream));
    S.drop_graphs();
    S.bytes -= S.wk_bytes;
    S.free_list(S.wk.allocs);
    S.wk.tG = S.wk.tW = S.wk.tA = S.wk.tM = S.wk.tS1 = S.wk.tS2 = TileSet();
    S.wk.tGb = S.wk.tGm = S.wk.tMb = S.wk.tMm = TileSet();
    const long long bytes_before = S.bytes;
    auto& w = S.wk;
    auto& L = w.allocs;
    const Geometry& g = S.g;
    const int m = S.restart;
    const long long ld = S.ld;
    const int nch = (int)((S.kp + kChunk - 1) / kChunk);
    const int rch = (int)((g.r + kChunk - 1) / kChunk);
    w.b = S.dalloc<double>((size_t)R * g.r, L);
    w.t2 = S.dalloc<double>((size_t)R * g.r, L);
    w.fstage = S.dalloc<double>((size_t)R * g.r, L);
    w.ustage = S.dalloc<double>((size_t)R * g.r, L);
    w.gstage = S.dalloc<double>((size_t)R * (2 * g.fz + 2 * g.nx), L);
    if (S.fss) {
        w.fs1 = S.dalloc<double>((size_t)R * g.r, L);
        w.fs2 = S.dalloc<double>((size_t)R * g.r, L);
        w.fs3 = S.dalloc<double>((size_t)R * g.r, L);
        w.k2r = S.dalloc<double>((size_t)R, L);
    }
    double** vecs[] = {&w.bS, &w.Xp, &w.t, &w.s, &w.w, &w.z, &w.xS, &w.xSlo, &w.slo, &w.sxlo};
    for (double** v : vecs) {
        *v = S.dalloc<double>((size_t)R * ld, L);
        k_fill(*v, (long long)R * ld, 0.0, S.stream);
    }
    w.V = S.dalloc<double>((size_t)R * (m + 1) * ld, L);
    k_fill(w.V, (long long)R * (m + 1) * ld, 0.0, S.stream);
    if (S.precision >= 1) {
        w.Zb = S.dalloc<double>((size_t)R * m * ld, L);
        k_fill(w.Zb, (long long)R * m * ld, 0.0, S.stream);
    }
    if (S.precision == 2) {
        const int mi = S.inner_m;
        w.Vi = S.dalloc<double>((size_t)R * (mi + 1) * ld, L);
        k_fill(w.Vi, (long long)R * (mi + 1) * ld, 0.0, S.stream);
        w.Hci = S.dalloc<double>((size_t)R * mi * (mi + 1), L);
        w.htmpi = S.dalloc<double>((size_t)R * (mi + 1), L);
        w.csi = S.dalloc<double>((size_t)R * mi, L);
        w.sni = S.dalloc<double>((size_t)R * mi, L);
        w.gvi = S.dalloc<double>((size_t)R * (mi + 1), L);
        w.part1i = S.dalloc<double>((size_t)R * nch * (mi + 2), L);
        w.part2i = S.dalloc<double>((size_t)R * nch * (mi + 2), L);
        w.qi = S.dalloc<double>((size_t)R * g.d, L);
        w.ci = S.dalloc<double>((size_t)R * g.d, L);
        w.c0i = S.dalloc<double>((size_t)R * g.d, L);
        w.targeti = S.dalloc<double>(R, L);
        w.bnormi = S.dalloc<double>(R, L);
        w.rnormi = S.dalloc<double>(R, L);
        w.activei = S.dalloc<int>(R, L);
        w.donei = S.dalloc<int>(R, L);
        w.niti = S.dalloc<int>(R, L);
        w.flagsi = S.dalloc<int>(R, L);
        double** iv[] = {&w.wi, &w.zi, &w.xi, &w.ti, &w.si, &w.Xpi, &w.vin};
        for (double** v : iv) {
            *v = S.dalloc<double>((size_t)R * ld, L);
            k_fill(*v, (long long)R * ld, 0.0, S.stream);
        }
        CK(cudaMemsetAsync(w.flagsi, 0, R * sizeof(int), S.stream));
    }
    w.Hc = S.dalloc<double>((size_t)R * m * (m + 1), L);
    w.htmp = S.dalloc<double>((size_t)R * (m + 1), L);
    w.cs = S.dalloc<double>((size_t)R * m, L);
    w.sn = S.dalloc<double>((size_t)R * m, L);
    w.gv = S.dalloc<double>((size_t)R * (m + 1), L);
    w.part1 = S.dalloc<double>((size_t)R * nch * (m + 2), L);
    w.part2 = S.dalloc<double>((size_t)R * nch * (m + 2), L);
    w.rpart = S.dalloc<double>((size_t)R * std::max(nch, rch), L);
    w.q = S.dalloc<double>((size_t)R * g.d, L);
    w.c = S.dalloc<double>((size_t)R * g.d, L);
    w.c0 = S.dalloc<double>((size_t)R * g.d, L);
    w.active = S.dalloc<int>(R, L);
    w.done = S.dalloc<int>(R, L);
    w.nit = S.dalloc<int>(R, L);
    w.hist = S.dalloc<double>((size_t)R * (S.max_iter + 1), L);
    w.hist_base = S.dalloc<int>(R, L);
    w.flags = S.dalloc<int>(R, L);
    w.op = S.dalloc<int>(R, L);
    w.gauge = S.dalloc<int>(R, L);
    w.target = S.dalloc<double>(R, L);
    w.bnorm = S.dalloc<double>(R, L);
    w.rnorm = S.dalloc<double>(R, L);
    w.uLp = (const double**)S.dalloc<double*>(R, L);
    w.uSp = (const double**)S.dalloc<double*>(R, L);
    w.oneSp = (const double**)S.dalloc<double*>(R, L);
    // tile lists sized for the worst case (every rhs its own op): units * R
    w.tG = w.tW = w.tA = w.tM = w.tS1 = w.tS2 = TileSet();   // built by prepare_ops
    w.tGb = w.tGm = w.tMb = w.tMm = TileSet();
    CK(cudaStreamSynchronize(S.stream));
    S.wk_bytes = S.bytes - bytes_before;
    S.Rcap = R;
    S.cur_ops.clear();
}

static std::vector<Tile> make_tiles(const std::vector<int>& unit_cls, int ncls, const std::vector<int>& ops, int bn) {
    std::vector<Tile> out;
    const int R = (int)ops.size(), nu = (int)unit_cls.size();
    int rb = 0;
    while (rb < R) {
        int re = rb;
        while (re < R && ops[re] == ops[rb]) ++re;
        int ub = 0;
        while (ub < nu) {
            int ue = ub;
            while (ue < nu && unit_cls[ue] == unit_cls[ub]) ++ue;
            for (int rr = rb; rr < re && unit_cls[ub] >= 0;) {   // class -1: units left out
                const int nr = std::min(bn, re - rr);
                const int upt = std::max(1, bn / nr);
                for (int u = ub; u < ue; u += upt)
                    out.push_back(Tile{ops[rb] * ncls + unit_cls[ub], u, std::min(upt, ue - u), rr, nr});
                rr += nr;
            }
            ub = ue;
        }
        rb = re;
    }
    return out;
}

static std::vector<Tile> make_slot_tiles(const Solver& S, const std::vector<int>& ops, int sz, int bn) {
    std::vector<Tile> out;
    const int R = (int)ops.size(), nu = (int)S.strip_cls.size();
    const int ns = std::max(sz == 1 ? S.ns1 : S.ns2, 1);
    int rb = 0;
    while (rb < R) {
        int re = rb;
        while (re < R && ops[re] == ops[rb]) ++re;
        int ub = 0;
        while (ub < nu) {
            int ue = ub;
            while (ue < nu && S.strip_cls[ue] == S.strip_cls[ub]) ++ue;
            const int c = S.strip_cls[ub];
            for (size_t t = 0; t < S.sl_size[c].size(); ++t) {
                if (S.sl_size[c][t] != sz) continue;
                const int mat = (ops[rb] * 3 + S.slot_cls[c]) * ns + S.sl_idx[c][t];
                const long long off = (long long)S.sl_start[c][t] * S.g.fz;
                for (int rr = rb; rr < re;) {
                    const int nr = std::min(bn, re - rr);
                    const int upt = std::max(1, bn / nr);
                    for (int u = ub; u < ue; u += upt) out.push_back(Tile{mat, u, std::min(upt, ue - u), rr, nr, off});
                    rr += nr;
                }
            }
            ub = ue;
        }
        rb = re;
    }
    return out;
}

// Upload a tile list of shape sh into ts (grown in the workspace as needed; a
// replaced list stays allocated until the workspace is freed).  The host
// vector must live until the stream has consumed the copy.
static void upload_tiles(Solver& S, TileSet& ts, int sh, const std::vector<Tile>& v) {
    if (v.size() > ts.cap || ts.t[sh] == nullptr) {
        const size_t cap = std::max<size_t>(v.size(), 1) * 2;
        for (int k = 0; k < 2; ++k) {   // both shapes share one capacity (shape 1 never has more tiles)
            Tile* fresh = S.dalloc<Tile>(cap, S.wk.allocs);
            if (ts.t[k] && k != sh && ts.n[k] > 0)
                CK(cudaMemcpyAsync(fresh, ts.t[k], ts.n[k] * sizeof(Tile), cudaMemcpyDeviceToDevice, S.stream));
            ts.t[k] = fresh;
        }
        ts.cap = cap;
    }
    if (!v.empty()) CK(cudaMemcpyAsync(ts.t[sh], v.data(), v.size() * sizeof(Tile), cudaMemcpyHostToDevice, S.stream));
    ts.n[sh] = (int)v.size();
}

static void prepare_ops(Solver& S, const std::vector<int>& ops) {
    if (ops == S.cur_ops) return;
    S.drop_graphs();
    auto& w = S.wk;
    std::vector<std::vector<Tile>> keep;   // host lists alive until the sync below
    for (int sh = 0; sh < 2; ++sh) {
        const int bn = gemm_tile_columns(sh);
        if (S.fss)
            for (int sz = 1; sz <= 2; ++sz) {
                keep.push_back(make_slot_tiles(S, ops, sz, bn));
                upload_tiles(S, sz == 1 ? w.tS1 : w.tS2, sh, keep.back());
            }
        keep.push_back(make_tiles(S.strip_cls, 3, ops, bn));
        upload_tiles(S, w.tG, sh, keep.back());
        upload_tiles(S, w.tW, sh, keep.back());
        upload_tiles(S, w.tA, sh, keep.back());
        keep.push_back(make_tiles(S.pair_mc, S.nmc, ops, bn));
        upload_tiles(S, w.tM, sh, keep.back());
        // mirror form: interior units in one list (matrix index = operator),
        // the other classes in another
        auto split = [&](const std::vector<int>& cls, int ncls, int mc, TileSet& tb, TileSet& tm) {
            std::vector<int> cb(cls), cm(cls);
            for (size_t u = 0; u < cls.size(); ++u) {
                cb[u] = cls[u] == mc ? -1 : cls[u];
                cm[u] = cls[u] == mc ? 0 : -1;
            }
            keep.push_back(make_tiles(cb, ncls, ops, bn));
            upload_tiles(S, tb, sh, keep.back());
            keep.push_back(make_tiles(cm, 1, ops, bn));
            upload_tiles(S, tm, sh, keep.back());
        };
        if (S.mirG) split(S.strip_cls, 3, 1, w.tGb, w.tGm);
        if (S.mirM) split(S.pair_mc, S.nmc, S.mc_int, w.tMb, w.tMm);
    }
    // The mirror form of S and M^-1 adds a launch for the boundary classes
    // (~10 us); it pays where it saves more than ~25 MFLOP per product
    // (256x4 order 12: 0.43 vs 0.59 ms for S x at 128 right-hand sides; an
    // 8x2 order-8 single solve: 1.06 vs 0.86 ms).
    {
        const double fz2 = (double)S.g.fz * S.g.fz, R = (double)ops.size();
        const double saveG = (double)(S.g.mx - 2) * R * 4.0 * fz2;
        int npi = 0;
        for (int mc : S.pair_mc) npi += mc == S.mc_int ? 1 : 0;
        const double saveM = (double)npi * R * 16.0 * fz2;
        S.useG = S.mirG && (S.mirror_mode == 1 || saveG >= 2.5e7);
        S.useM = S.mirM && (S.mirror_mode == 1 || saveM >= 2.5e7);
    }
    const int R = (int)ops.size();
    std::vector<const double*> uLp(R, nullptr), uSp(R, nullptr), oneSp(R, nullptr);
    std::vector<int> gauge(R, 0);
    for (int r = 0; r < R; ++r)
        if (ops[r] == S.singular_op) {
            uLp[r] = S.uL;
            uSp[r] = S.uS;
            oneSp[r] = S.oneS;
            gauge[r] = 1;
        }
    CK(cudaMemcpyAsync(w.op, ops.data(), R * sizeof(int), cudaMemcpyHostToDevice, S.stream));
    if (S.fss) {
        std::vector<double> k2r(R);
        for (int r = 0; r < R; ++r) k2r[r] = S.k2[ops[r]];
        CK(cudaMemcpyAsync(w.k2r, k2r.data(), R * sizeof(double), cudaMemcpyHostToDevice, S.stream));
        CK(cudaStreamSynchronize(S.stream));
    }
    CK(cudaMemcpyAsync(w.gauge, gauge.data(), R * sizeof(int), cudaMemcpyHostToDevice, S.stream));
    CK(cudaMemcpyAsync(w.uLp, uLp.data(), R * sizeof(double*), cudaMemcpyHostToDevice, S.stream));
    CK(cudaMemcpyAsync(w.uSp, uSp.data(), R * sizeof(double*), cudaMemcpyHostToDevice, S.stream));
    CK(cudaMemcpyAsync(w.oneSp, oneSp.data(), R * sizeof(double*), cudaMemcpyHostToDevice, S.stream));
    CK(cudaStreamSynchronize(S.stream));
    S.cur_ops = ops;
}

// ---------------------------------------------------------------------------
// Solve
// ---------------------------------------------------------------------------

static bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static GemmArgs gemm_base(const Solver& S) {
    GemmArgs a;
    std::memset(&a, 0, sizeof(a));
    (void)S;
    return a;
}

static constexpr int kEventPairs = 8192;

// Tile-shape autotuner.  The first time a GEMM of a given kind (epilogue,
// precision, M, K, size class of the column count) runs outside a graph
// capture and outside profiling, both tile shapes are launched twice each on
// the real operands (every launch writes the complete output, so the result
// stands), timed with CUDA events, and the faster shape is kept for that key
// for the rest of the process (all handles, all threads).
static std::mutex g_tune_mu;
static std::map<std::array<int, 7>, int> g_tune;

static std::array<int, 7> tune_key(const GemmArgs& a, const TileSet& ts, int epi) {
    int dev = 0;
    cudaGetDevice(&dev);
    int bucket = 0;
    while ((1 << (bucket + 1)) <= ts.n[0]) ++bucket;
    return {dev, epi, a.fp32, a.M, a.K, bucket, a.mirror_nb};
}

static int tune_shape(Solver& S, GemmArgs& a, const TileSet& ts, int epi, bool& launched) {
    launched = false;
    if (ts.n[1] <= 0 || epi == 3) return 0;
    const std::array<int, 7> key = tune_key(a, ts, epi);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    if (S.capturing || S.prof) return 0;
    cudaEvent_t e[5];
    for (auto& x : e) CK(cudaEventCreate(&x));
    CK(cudaEventRecord(e[0], S.stream));
    for (int rep = 0; rep < 2; ++rep)
        for (int sh = 0; sh < 2; ++sh) {
            a.shape = sh;
            launch_class_gemm(a, ts.t[sh], ts.n[sh], epi, S.stream);
            CK(cudaEventRecord(e[1 + rep * 2 + sh], S.stream));
        }
    CK(cudaEventSynchronize(e[4]));
    float t[4];
    CK(cudaEventElapsedTime(&t[0], e[0], e[1]));
    for (int k = 1; k < 4; ++k) CK(cudaEventElapsedTime(&t[k], e[k], e[k + 1]));
    for (auto& x : e) cudaEventDestroy(x);
    const int best = std::min(t[1], t[3]) < std::min(t[0], t[2]) ? 1 : 0;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune.emplace(key, best);
    }
    launched = true;
    return best;
}

static void run_gemm(Solver& S, GemmArgs a, const TileSet& ts, int epi) {
    if (S.oz && !S.capturing_prof_block() && (S.oz_mask & (a.fp32 ? 2 : 1)) && a.mirror_nb == 0 &&
        (epi == 0 || epi == 1)) {
        auto it = S.ozmats.find(a.mats);
        if (it != S.ozmats.end()) {
            const Solver::OzMat& m = it->second;
            const int sh = m.N == 64 ? 1 : 0;     // tile lists of 64 or 32 columns
            OzArgs z;
            z.a = a;
            z.dig = m.dig; z.dig_stride = m.dig_stride; z.rexp = m.rexp; z.rexp_stride = m.rexp_stride;
            z.S = m.S; z.beta = m.beta; z.N = m.N; z.mt_n = m.mt_n; z.kcn = m.kcn; z.epi = epi; z.err = S.d_ozerr;
            const bool rec = S.prof && S.ev_used < kEventPairs;
            if (S.prof) z.a.flops = S.d_flops + 2;       // [2] algorithmic, [3] executed tensor FLOPs
            if (rec) {
                S.ev_f32[S.ev_used] = 2;
                CK(cudaEventRecord(S.ev[2 * S.ev_used], S.stream));
            }
            const bool ok = launch_oz_gemm(z, ts.t[sh], ts.n[sh], S.stream);
            if (rec) {
                CK(cudaEventRecord(S.ev[2 * S.ev_used + 1], S.stream));
                ++S.ev_used;
            }
            if (ok) return;
            cudaGetLastError();
            S.oz = false;                        // SIMT products from now on
            S.oz_mask = 0;
        }
    }
    bool launched = false;
    const int sh = std::getenv("SMPM_TILE_SHAPE") ? std::atoi(std::getenv("SMPM_TILE_SHAPE")) & 1
                                                  : tune_shape(S, a, ts, epi, launched);
    if (launched) return;                // the tuning launches computed the output
    a.shape = sh;
    const Tile* tiles = ts.t[sh];
    const int ntiles = ts.n[sh];
    if (S.prof && S.cap_events) {   // inside a graph capture: the graph owns its events
        a.flops = S.d_flops + (a.fp32 ? 1 : 0);
        S.cap_f32->push_back(a.fp32 ? 1 : 0);
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        S.cap_events->push_back(e0);
        S.cap_events->push_back(e1);
        // external records: real event-record nodes of the graph (a plain
        // record inside a capture only orders the captured work)
        CK(cudaEventRecordWithFlags(e0, S.stream, cudaEventRecordExternal));
        launch_class_gemm(a, tiles, ntiles, epi, S.stream);
        CK(cudaEventRecordWithFlags(e1, S.stream, cudaEventRecordExternal));
        return;
    }
    const bool rec = S.prof && S.ev_used < kEventPairs;
    if (S.prof) a.flops = S.d_flops + (a.fp32 ? 1 : 0);
    if (rec) {
        S.ev_f32[S.ev_used] = a.fp32 ? 1 : 0;
        CK(cudaEventRecord(S.ev[2 * S.ev_used], S.stream));
    }
    launch_class_gemm(a, tiles, ntiles, epi, S.stream);
    if (rec) {
        CK(cudaEventRecord(S.ev[2 * S.ev_used + 1], S.stream));
        ++S.ev_used;
    }
}

// Tile shape a launch of this kind uses (tuning it now, on the real
// operands, if it has not been tuned in this process yet).
static int shape_for(Solver& S, const GemmArgs& a, const TileSet& ts, int epi) {
    if (const char* e = std::getenv("SMPM_TILE_SHAPE")) return std::atoi(e) & 1;
    if (ts.n[1] <= 0 || epi == 3) return 0;
    const std::array<int, 7> key = tune_key(a, ts, epi);
    for (int pass = 0; pass < 2; ++pass) {
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) return it->second;
        }
        if (pass == 0) run_gemm(S, a, ts, epi);
    }
    return 0;
}

// One dense-product launch (arguments, tile lists, epilogue).
struct GemmCall {
    GemmArgs a;
    const TileSet* ts;
    int epi;
};

static PGemm to_pgemm(Solver& S, const GemmCall& c) {
    const int sh = shape_for(S, c.a, *c.ts, c.epi);
    const int bm = sh == 1 ? 8 : 16;
    PGemm g;
    g.a = c.a;
    g.a.shape = sh;
    g.tiles = c.ts->t[sh];
    g.ntiles = c.ts->n[sh];
    g.nrow = (c.a.M + bm - 1) / bm;
    g.epi = c.epi;
    return g;
}

// Process-wide profile totals (every handle's harvested launches; per
// precision: [0] FP64, [1] FP32), and whether new handles profile.
static std::mutex g_prof_mu;
static long long g_prof_launches[4] = {0, 0, 0, 0};
static double g_prof_ms[4] = {0.0, 0.0, 0.0, 0.0}, g_prof_flops[4] = {0.0, 0.0, 0.0, 0.0};
static std::atomic<int> g_prof_default{0};

static void add_prof(Solver& S, int p, long long n, double ms, double flops) {
    S.prof_launches[p] += n;
    S.prof_ms[p] += ms;
    S.prof_flops[p] += flops;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_launches[p] += n;
    g_prof_ms[p] += ms;
    g_prof_flops[p] += flops;
}

// Accumulate the recorded GEMM launches (after the stream has drained).
static void harvest_profile(Solver& S) {
    if (!S.prof) return;
    for (int i = 0; i < S.ev_used; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, S.ev[2 * i], S.ev[2 * i + 1]));
        add_prof(S, S.ev_f32[i], 1, ms, 0.0);
    }
    S.ev_used = 0;
    unsigned long long fl[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(fl, S.d_flops, sizeof(fl), cudaMemcpyDeviceToHost));
    for (int p = 0; p < 4; ++p) add_prof(S, p, 0, 0.0, (double)fl[p]);
    CK(cudaMemset(S.d_flops, 0, sizeof(fl)));
}

// Schur product out = add + sum_i scatter_i G_i gather_i in (Sec. 3.1,
// assembled blocks) with the FP64 blocks or their FP32 copies; the interior
// strips go through the mirror form when the handle has it.
static int schur_calls(Solver& S, const double* in, long long in_rs, long long in_off, double* out,
                       const double* add, const int* active, bool fp32, GemmCall* c) {
    const int fz = S.g.fz, f2 = 2 * fz;
    GemmArgs a = gemm_base(S);
    a.mats = fp32 ? reinterpret_cast<const double*>(S.G32) : S.G;
    a.fp32 = fp32 ? 1 : 0;
    a.mat_stride = S.sG; a.M = f2; a.K = f2;
    a.row_lo = S.rl_GW; a.row_hi = S.rh_GW;
    a.in = in; a.in_rs = in_rs; a.in_us = f2; a.in_off = in_off;
    a.out = out; a.out_rs = S.ld; a.out_us = f2; a.out_off0 = -fz; a.out_off1 = f2; a.msplit = fz;
    a.add = add;
    a.active = active;
    const double* h = fp32 ? reinterpret_cast<const double*>(S.Gh32) : S.Gh;
    if (!S.useG || h == nullptr || (S.oz_mask & (fp32 ? 2 : 1))) {
        c[0] = GemmCall{a, &S.wk.tG, 1};
        return 1;
    }
    c[0] = GemmCall{a, &S.wk.tGb, 1};
    a.mats = h; a.mat_stride = 2LL * fz * fz; a.M = a.K = fz; a.mirror_nb = 2; a.face = fz;
    c[1] = GemmCall{a, &S.wk.tGm, 1};
    return 2;
}

static void schur_product(Solver& S, const double* in, long long in_rs, long long in_off, double* out,
                          const double* add, const int* active, bool fp32) {
    GemmCall c[2];
    const int n = schur_calls(S, in, in_rs, in_off, out, add, active, fp32, c);
    for (int i = 0; i < n; ++i) run_gemm(S, c[i].a, *c[i].ts, c[i].epi);
}

// Block-Jacobi apply out = M_p^-1 in over the pairs p (faces [(4p+1) fz,
// (4p+5) fz), Sec. 3.2); the interior pairs through the mirror form when the
// handle has it.
static int bj_calls(Solver& S, const double* in, long long in_rs, long long in_off, double* out, long long out_rs,
                    long long out_off, const int* active, bool fp32, GemmCall* c) {
    const int fz = S.g.fz, f4 = 4 * fz;
    GemmArgs a = gemm_base(S);
    a.mats = fp32 ? reinterpret_cast<const double*>(S.Minv32) : S.Minv;
    a.fp32 = fp32 ? 1 : 0;
    a.mat_stride = S.sM; a.M = f4; a.K = f4;
    a.row_lo = S.rl_M; a.row_hi = S.rh_M;
    a.in = in; a.in_rs = in_rs; a.in_us = f4; a.in_off = in_off + fz;
    a.out = out; a.out_rs = out_rs; a.out_us = f4; a.out_off0 = out_off + fz; a.out_off1 = 0; a.msplit = f4;
    a.active = active;
    const double* h = fp32 ? reinterpret_cast<const double*>(S.Mh32) : S.Mh;
    if (!S.useM || h == nullptr || (S.oz_mask & (fp32 ? 2 : 1))) {
        c[0] = GemmCall{a, &S.wk.tM, 0};
        return 1;
    }
    c[0] = GemmCall{a, &S.wk.tMb, 0};
    a.mats = h; a.mat_stride = 8LL * fz * fz; a.M = a.K = 2 * fz; a.mirror_nb = 4; a.face = fz;
    c[1] = GemmCall{a, &S.wk.tMm, 0};
    return 2;
}

static void bj_apply(Solver& S, const double* in, long long in_rs, long long in_off, double* out, long long out_rs,
                     long long out_off, const int* active, bool fp32) {
    GemmCall c[2];
    const int n = bj_calls(S, in, in_rs, in_off, out, out_rs, out_off, active, fp32, c);
    for (int i = 0; i < n; ++i) run_gemm(S, c[i].a, *c[i].ts, c[i].epi);
}

static int solve_impl(Solver& S, const std::vector<int>& ops, const double* f, const double* gb, double tol,
                      double* u, smpm_stats* st, const double* u0 = nullptr) {
    NvtxRange nvtx_range("smpm solve");
    auto t0 = std::chrono::steady_clock::now();
    const int R = (int)ops.size();
    if (R <= 0) throw Err{SMPM_EINVAL, "nrhs must be positive"};
    if (!(tol > 0.0)) throw Err{SMPM_EINVAL, "tol must be positive"};
    if (!f || !u) throw Err{SMPM_EINVAL, "f and u must not be null"};
    // SMPM_TRACE_PHASES=1: wall time of the solve's phases on stderr (the
    // stream is synchronised at every phase boundary, so this slows the solve)
    const bool tphase = std::getenv("SMPM_TRACE_PHASES") != nullptr;
    auto tp_last = std::chrono::steady_clock::now();
    std::string tp_msg;
    auto phase = [&](const char* name) {
        if (!tphase) return;
        CK(cudaStreamSynchronize(S.stream));
        const auto now = std::chrono::steady_clock::now();
        char buf[96];
        snprintf(buf, sizeof(buf), " %s=%.2f", name, std::chrono::duration<double, std::milli>(now - tp_last).count());
        tp_msg += buf;
        tp_last = now;
    };
    ensure_workspace(S, R);
    phase("workspace");
    prepare_ops(S, ops);
    phase("tiles");
    const Geometry& g = S.g;
    auto& w = S.wk;
    cudaStream_t st_ = S.stream;
    const int fz = g.fz, n = g.n, nfz = n * fz, f2 = 2 * fz, f4 = 4 * fz, m = S.restart;
    const long long ld = S.ld, nb = 2LL * fz + 2LL * g.nx;
    const int nch = (int)((S.kp + kChunk - 1) / kChunk);
    const int rch = (int)((g.r + kChunk - 1) / kChunk);

    // inputs
    const double* f_d = f;
    if (!is_device_ptr(f)) {
        CK(cudaMemcpyAsync(w.fstage, f, sizeof(double) * g.r * R, cudaMemcpyHostToDevice, st_));
        f_d = w.fstage;
    }
    const double* g_d = gb;
    if (gb && !is_device_ptr(gb)) {
        CK(cudaMemcpyAsync(w.gstage, gb, sizeof(double) * nb * R, cudaMemcpyHostToDevice, st_));
        g_d = w.gstage;
    }
    const bool u_dev = is_device_ptr(u);
    double* u_d = u_dev ? u : w.ustage;

    GridArgs ga;
    ga.n = n; ga.N = g.N; ga.mx = g.mx; ga.mz = g.mz; ga.fz = fz; ga.nx = g.nx; ga.r = g.r;
    ga.tau_x = g.tau_x; ga.tau_z = S.d_tau_z; ga.wq = S.d_wq; ga.hz = S.d_hz; ga.hx = g.hx; ga.area = g.lx * g.lz;

    // Alg. seq steps 1-3
    k_rhs_assemble(ga, R, f_d, g.r, g_d, nb, w.b, g.r, w.uLp, w.rpart, rch, kChunk, st_);
    k_project(R, g.r, w.b, g.r, w.uLp, w.rpart, rch, kChunk, st_);
    const FssArgs fa{n, fz, g.mx, S.d_strip_cls};
    if (S.fss) {  // b_S = B (A^-1 b): fast strip solves, then the face fluxes
        fss_refined(S, fa, R, w.b, g.r, w.t2, g.r, nullptr, 0, w.k2r, w.fs1, w.fs2, w.fs3, w.tS1, w.tS2);
        k_face_flux(fa, R, S.d_beta, w.t2, g.r, w.bS, ld, S.kp, st_);
    } else {
        GemmArgs aW = gemm_base(S);
        aW.mats = S.W; aW.mat_stride = S.sW; aW.M = f2; aW.K = nfz;
        aW.row_lo = S.rl_GW; aW.row_hi = S.rh_GW;
        aW.in = w.b; aW.in_rs = g.r; aW.in_us = nfz; aW.in_off = 0;
        aW.out = w.bS; aW.out_rs = ld; aW.out_us = f2; aW.out_off0 = -fz; aW.out_off1 = f2; aW.msplit = fz;
        run_gemm(S, aW, w.tW, 0);
    }
    // SMPM_TRACE_SOLVE=1: per-cycle true residual and iterate norms on stderr
    const bool trace = std::getenv("SMPM_TRACE_SOLVE") != nullptr;
    std::vector<double> tr_v;
    auto host_norms = [&](const double* v, const char* name) {
        tr_v.resize((size_t)R * ld);
        CK(cudaMemcpyAsync(tr_v.data(), v, sizeof(double) * tr_v.size(), cudaMemcpyDeviceToHost, st_));
        CK(cudaStreamSynchronize(st_));
        for (int r = 0; r < R; ++r) {
            double s2 = 0.0, s1 = 0.0;
            for (long long i = 0; i < S.kp; ++i) {
                const double x = tr_v[(size_t)r * ld + i];
                s2 += x * x;
                s1 += x;
            }
            fprintf(stderr, " %s[%d]: |v| %.3e sum %.3e", name, r, std::sqrt(s2), s1);
        }
    };
    if (trace) {
        fprintf(stderr, "smpm solve trace:");
        host_norms(w.bS, "bS_unprojected");
        fprintf(stderr, "\n");
    }
    k_dot_partial(R, S.kp, w.bS, ld, w.uSp, w.rpart, nch, kChunk, st_);
    k_project(R, S.kp, w.bS, ld, w.uSp, w.rpart, nch, kChunk, st_);
    if (trace) {
        fprintf(stderr, "smpm solve trace:");
        host_norms(w.bS, "bS");
        fprintf(stderr, "\n");
    }

    phase("rhs");
    KArgs ka;
    std::memset(&ka, 0, sizeof(ka));
    ka.R = R; ka.m = m; ka.nch = nch; ka.ch = kChunk; ka.ld = ld; ka.kp = S.kp;
    ka.fz = fz; ka.mx = g.mx; ka.ng = g.ng; ka.d = g.d; ka.n = n;
    ka.V = w.V; ka.w = w.w; ka.Hc = w.Hc; ka.htmp = w.htmp; ka.cs = w.cs; ka.sn = w.sn; ka.gv = w.gv;
    ka.part1 = w.part1; ka.part2 = w.part2; ka.q = w.q; ka.c = w.c;
    ka.rho = S.rho; ka.rho_stride = S.sRho; ka.K = S.K; ka.K_stride = S.sK;
    ka.op = w.op; ka.strip_cls = S.d_strip_cls;
    ka.active = w.active; ka.done = w.done; ka.nit = w.nit; ka.target = w.target;
    ka.bnorm = w.bnorm; ka.rnorm = w.rnorm; ka.flags = w.flags;
    ka.grp = S.krylov == 1 ? R : 1;
    ka.hist = w.hist; ka.hist_base = w.hist_base; ka.hist_stride = S.max_iter + 1;

    // Nested mixed-precision form (precision 2): the outer flexible GMRES runs
    // on S itself (no deflation: K = null makes every coarse coefficient zero)
    // and its preconditioner is an inner DBJ-GMRES with FP32 Schur blocks and
    // FP32 block-Jacobi, inner_m steps or 1e-4 relative, from a zero guess.
    const bool nested = S.precision == 2;
    KArgs ki = ka;
    if (nested) {
        ki.m = S.inner_m;
        ki.V = w.Vi; ki.w = w.wi; ki.Hc = w.Hci; ki.htmp = w.htmpi; ki.cs = w.csi; ki.sn = w.sni; ki.gv = w.gvi;
        ki.part1 = w.part1i; ki.part2 = w.part2i; ki.q = w.qi; ki.c = w.ci;
        ki.active = w.activei; ki.done = w.donei; ki.nit = w.niti; ki.target = w.targeti;
        ki.bnorm = w.bnormi; ki.rnorm = w.rnormi; ki.flags = w.flagsi;
        ki.f32 = std::getenv("SMPM_INNER_FP64_ARNOLDI") ? 0 : 1;
        ki.hist = nullptr;                       // the history is the outer iteration's
        ka.K = nullptr;
    }

    // block-Jacobi apply: out = Minv_p in over pairs p (faces [(4p+1) fz, (4p+5) fz))
    auto bj = [&](const double* in, long long in_rs, long long in_off, double* out, long long out_rs,
                  long long out_off, const int* active, bool fp32 = false) {
        bj_apply(S, in, in_rs, in_off, out, out_rs, out_off, active, fp32);
    };
    // Schur product: out = in + sum_i scatter_i G_i gather_i in
    // (identity term from the same layout when in_rs == ld and in_off == 0)
    auto schur = [&](const double* in, long long in_rs, long long in_off, double* out, const int* active) {
        schur_product(S, in, in_rs, in_off, out, in, active, false);
    };
    // FP32 Schur product of the inner solve (FP32 blocks and accumulation)
    auto schur32 = [&](const double* in, double* out, const int* active) {
        schur_product(S, in, ld, 0, out, in, active, true);
    };
    // z = inner solve of S z = V_j for the active right-hand sides (one
    // deflated right-preconditioned GMRES cycle from z = 0, Alg. seq steps
    // 4-8 with FP32 operators), result in w.xi
    auto inner_solve = [&](int jj) {
        const int mi = S.inner_m;
        CK(cudaMemcpy2DAsync(w.vin, (size_t)ld * 8, w.V + (long long)jj * ld, (size_t)(m + 1) * ld * 8,
                             (size_t)S.kp * 8, R, cudaMemcpyDeviceToDevice, st_));
        k_invert_flags(w.donei, w.active, R, st_);
        k_fill(w.xi, (long long)R * ld, 0.0, st_);
        k_residual(ki, w.vin, nullptr, st_);
        k_cycle_start(ki, w.c0i, 1, 1e-4, st_);
        for (int t = 0; t < mi; ++t) {
            bj(w.Vi, (long long)(mi + 1) * ld, (long long)t * ld, w.zi, ld, 0, w.activei, true);
            schur32(w.zi, w.wi, w.activei);
            k_deflate_sum(ki, w.wi, nullptr, st_);
            k_coarse(ki, st_);
            k_cgs(ki, t, 0, st_);
            k_cgs(ki, t, 1, st_);
            k_cgs(ki, t, 2, st_);
            k_normalize(ki, t, mi, st_);
        }
        k_cycle_update(ki, w.Xpi, st_);
        bj(w.Xpi, ld, 0, w.ti, ld, 0, nullptr, true);
        schur32(w.ti, w.si, nullptr);
        k_deflate_coarse_pending(ki, w.si, st_);
        k_xs_update(ki, w.xi, w.ti, w.c0i, st_);
    };
    // compensated Schur product of x_S (hi part in out, low part in out_lo)
    auto schur_ext = [&](const double* in, double* out, double* out_lo) {
        GemmArgs a = gemm_base(S);
        a.mats = S.G; a.mat_stride = S.sG; a.M = f2; a.K = f2;
        a.row_lo = S.rl_GW; a.row_hi = S.rh_GW;
        a.in = in; a.in_rs = ld; a.in_us = f2; a.in_off = 0;
        a.out = out; a.out_rs = ld; a.out_us = f2; a.out_off0 = -fz; a.out_off1 = f2; a.msplit = fz;
        a.add = in;
        a.out_lo = out_lo;
        run_gemm(S, a, w.tG, 3);
    };

    CK(cudaMemsetAsync(w.done, 0, R * sizeof(int), st_));
    CK(cudaMemsetAsync(w.active, 0, R * sizeof(int), st_));
    CK(cudaMemsetAsync(w.flags, 0, R * sizeof(int), st_));
    CK(cudaMemsetAsync(w.nit, 0, R * sizeof(int), st_));
    k_fill(w.xS, (long long)R * ld, 0.0, st_);
    // warm start: x_S0 = B u0 (the interface unknowns of a guess, Sec. 2.3:
    // the exact solution has x_S = B u)
    const bool warm = u0 != nullptr && S.fss;
    if (warm) {
        const double* u0_d = u0;
        if (!is_device_ptr(u0)) {
            CK(cudaMemcpyAsync(w.ustage, u0, sizeof(double) * g.r * R, cudaMemcpyHostToDevice, st_));
            u0_d = w.ustage;
        }
        k_face_flux(fa, R, S.d_beta, u0_d, g.r, w.xS, ld, S.kp, st_);
    }

    // Restart cycles as iterative refinement on x_S: every cycle starts from the
    // true residual d = b_S - S x_S, runs deflated right-preconditioned GMRES on
    // P S M^-1 y = P d, and adds dx = t + Z K Z^T (d - S t), t = M^-1 V y
    // (= Q M^-1 y + Z C\ d of Eq. deflated_schur for this cycle's system).
    std::vector<int> h_done(R), h_active(R), h_nit(R), h_flags(R);
    // Stagnation of the refinement: a right-hand side whose true residual is
    // already within 1e3 tol and drops by less than 2x in two consecutive
    // cycles has reached the FP64 floor of ||S x_S - b_S|| (rounding of the
    // Schur product, ~ eps |G| |x_S|); it stops there with SMPM_ENOCONV instead
    // of running to max_iter.
    std::vector<double> prev_rel(R, -1.0), h_rn(R), h_bn(R);
    std::vector<int> stall(R, 0);
    // residual history: the true residual at every cycle start of a
    // right-hand side still running, and the Arnoldi steps taken so far
    // (each step's Givens estimate is written by the normalisation kernel)
    std::vector<int> h_base(R, 0), was_done(R, 0);
    S.hist_true.assign(R, std::vector<double>());
    S.hist_R = 0;
    const int one_i = 1, zero_i = 0;
    bool stagnated = false;
    int total_it = 0, cycles = 0, status = SMPM_OK;
    bool first = true;
    const int check_every = 4;
    const bool graphs_off = std::getenv("SMPM_NO_GRAPHS") != nullptr;
    // SMPM_PERSISTENT=1: the Arnoldi steps of a cycle in one persistent
    // cooperative kernel instead of step groups of separate launches
    // (graph-replayed), which measured 5-7 % faster on GB300 (256 x 4, order
    // 12, 128 right-hand sides: 40.3 vs 42.4-43.5 ms per batch; 8 x 2, order
    // 8: 857 vs 902 us per solve); SMPM_PERSIST_WAIT_NS: time limit of a
    // barrier wait (default 2 s); SMPM_PERSIST_STALL=1: test hook, every
    // barrier waits for a block that does not exist, so the first wait runs
    // out of time and the solve returns SMPM_ETIMEOUT
    const char* pe = std::getenv("SMPM_PERSISTENT");
    const bool persist_off = pe == nullptr || std::atoi(pe) == 0;
    const char* pw = std::getenv("SMPM_PERSIST_WAIT_NS");
    const long long persist_wait_ns = pw ? std::max(1000LL, std::atoll(pw)) : 2000000000LL;
    const bool persist_stall = std::getenv("SMPM_PERSIST_STALL") != nullptr;
    // Extended-precision refinement: when the true residual stalls near tol
    // (the FP64 rounding floor of S x_S, ~ eps |G| |x_S|, reached when |x_S| is
    // far above |b_S|), the iterate is kept as x_S + x_lo (double-double), and
    // the cycle-start residual b_S - S (x_S + x_lo) is formed with the
    // compensated Schur product; the GMRES cycles themselves stay FP64
    // (iterative refinement with an extra-precise residual).
    // precision 1 applies the block-Jacobi blocks in FP32; when a refinement
    // cycle reduces the true residual by less than 10x (FP32 blocks too coarse
    // for an ill-conditioned M, e.g. large k^2), the remaining cycles of this
    // solve use the FP64 blocks (the flexible GMRES allows the switch)
    bool bj_fp32 = S.precision == 1 && S.bj32_ok;
    bool group_fp32 = bj_fp32;
    double prev_cycle_rel = -1.0;
    bool ext = false;
    if (std::getenv("SMPM_REFINE_EXTENDED") != nullptr) {   // from the first refinement step on
        ext = true;
        k_fill(w.xSlo, (long long)R * ld, 0.0, st_);
        ka.xlo = w.xSlo;
        ka.s_lo = w.slo;
        ka.s_xlo = w.sxlo;
    }
    auto cycle_residual = [&](bool zero_x, bool stamp) {
        if (!zero_x) {
            if (ext) {
                schur_ext(w.xS, w.s, w.slo);
                schur(w.xSlo, ld, 0, w.sxlo, nullptr);
            } else {
                schur(w.xS, ld, 0, w.s, nullptr);
            }
            // k^2 = 0: b_S is projected out of u_S (Eq. regularize_schur), so the
            // residual is taken in the same complement: d = (I - u_S u_S^T)(b_S - S x_S).
            // The stored S (G from rounded strip solves) has u_S as left null
            // vector only to ~1e-13 |S|; without this the u_S component of S x_S,
            // ~1e-13 |S| |x_S|, is a residual floor no correction can reach
            // (2.3e-10 on 512 x 16, order 12, where |x_S| ~ 250 |b_S|).
            k_dot_partial(R, S.kp, w.s, ld, w.uSp, w.rpart, nch, kChunk, st_);
            k_project(R, S.kp, w.s, ld, w.uSp, w.rpart, nch, kChunk, st_);
        }
        k_residual(ka, w.bS, zero_x ? nullptr : w.s, st_);
        k_cycle_start(ka, w.c0, stamp ? 1 : 0, tol, st_);
    };
    while (true) {
        cycle_residual(first && !warm, first);
        CK(cudaMemcpyAsync(h_done.data(), w.done, R * sizeof(int), cudaMemcpyDeviceToHost, st_));
        CK(cudaMemcpyAsync(h_rn.data(), w.rnorm, R * sizeof(double), cudaMemcpyDeviceToHost, st_));
        CK(cudaMemcpyAsync(h_bn.data(), w.bnorm, R * sizeof(double), cudaMemcpyDeviceToHost, st_));
        CK(cudaStreamSynchronize(st_));
        for (int r = 0; r < R; ++r) {
            if (!was_done[r]) S.hist_true[r].push_back(h_bn[r] > 0.0 ? h_rn[r] / h_bn[r] : 0.0);
            was_done[r] = h_done[r];
        }
        if (trace) {
            fprintf(stderr, "smpm solve trace: cycle %d it %d", cycles, total_it);
            for (int r = 0; r < R; ++r) fprintf(stderr, " rel[%d] %.3e", r, h_bn[r] > 0 ? h_rn[r] / h_bn[r] : 0.0);
            host_norms(w.xS, "xS");
            fprintf(stderr, "\n");
        }
        if (bj_fp32 && !first) {
            double worst_rel = 0.0;
            for (int r = 0; r < R; ++r)
                if (!h_done[r] && h_bn[r] > 0.0) worst_rel = std::max(worst_rel, h_rn[r] / h_bn[r]);
            if (worst_rel > 0.0 && prev_cycle_rel > 0.0 && worst_rel > 0.1 * prev_cycle_rel) bj_fp32 = false;
            prev_cycle_rel = worst_rel;
        } else if (bj_fp32) {
            prev_cycle_rel = 1.0;
        }
        bool switch_ext = false;
        for (int r = 0; r < R; ++r) {
            if (h_done[r] || !(h_bn[r] > 0.0)) continue;
            const double rel = h_rn[r] / h_bn[r];
            stall[r] = (prev_rel[r] > 0.0 && rel > 0.5 * prev_rel[r] && rel < 1e3 * tol) ? stall[r] + 1 : 0;
            prev_rel[r] = rel;
            if (!ext && stall[r] >= 1) switch_ext = true;
        }
        if (switch_ext) {
            ext = true;
            k_fill(w.xSlo, (long long)R * ld, 0.0, st_);
            ka.xlo = w.xSlo;
            ka.s_lo = w.slo;
            ka.s_xlo = w.sxlo;
            std::fill(stall.begin(), stall.end(), 0);
            cycle_residual(false, false);   // this cycle starts from the extra-precise residual
            CK(cudaMemcpyAsync(h_done.data(), w.done, R * sizeof(int), cudaMemcpyDeviceToHost, st_));
            CK(cudaMemcpyAsync(h_rn.data(), w.rnorm, R * sizeof(double), cudaMemcpyDeviceToHost, st_));
            CK(cudaStreamSynchronize(st_));
            for (int r = 0; r < R; ++r)
                if (!h_done[r] && h_bn[r] > 0.0) prev_rel[r] = h_rn[r] / h_bn[r];
            if (trace) {
                fprintf(stderr, "smpm solve trace: extended residual");
                for (int r = 0; r < R; ++r) fprintf(stderr, " rel[%d] %.3e", r, h_bn[r] > 0 ? h_rn[r] / h_bn[r] : 0.0);
                fprintf(stderr, "\n");
            }
        }
        for (int r = 0; r < R; ++r) {
            if (h_done[r] || !(h_bn[r] > 0.0)) continue;
            if (ext && stall[r] >= 2) {
                CK(cudaMemcpyAsync(w.done + r, &one_i, sizeof(int), cudaMemcpyHostToDevice, st_));
                CK(cudaMemcpyAsync(w.active + r, &zero_i, sizeof(int), cudaMemcpyHostToDevice, st_));
                h_done[r] = 1;
                stagnated = true;
            }
        }
        bool all = true;
        for (int r = 0; r < R; ++r) all &= h_done[r] != 0;
        if (all) break;
        if (total_it >= S.max_iter) { status = SMPM_ENOCONV; break; }
        const int last_allowed = std::min(m, S.max_iter - total_it);
        CK(cudaMemcpyAsync(w.hist_base, h_base.data(), R * sizeof(int), cudaMemcpyHostToDevice, st_));
        int j = 0;
        const bool mixed = S.precision >= 1;      // flexible: the preconditioned vectors are kept
        // (the nested form's steps carry whole inner solves; they run uncaptured)
        const bool use_graphs = S.graphs_ok && !graphs_off && !nested;
        // one Arnoldi step j of every active right-hand side
        auto step = [&](int jj) {
            // z_j = M^-1 v_j (FP32 block-Jacobi in the mixed form, the inner
            // FP32 DBJ-GMRES in the nested form: the flexible variant keeps z_j,
            // so the cycle's correction is exactly sum y_j z_j)
            double* zj = w.z;
            if (nested) {
                inner_solve(jj);
                zj = w.xi;
            } else {
                bj(w.V, (long long)(m + 1) * ld, (long long)jj * ld, w.z, ld, 0, w.active, group_fp32);
            }
            if (mixed)
                CK(cudaMemcpy2DAsync(w.Zb + (long long)jj * ld, (size_t)m * ld * 8, zj, (size_t)ld * 8,
                                     (size_t)S.kp * 8, R, cudaMemcpyDeviceToDevice, st_));
            schur(zj, ld, 0, w.w, w.active);
            k_deflate_sum(ka, w.w, nullptr, st_);
            k_coarse(ka, st_);
            k_cgs(ka, jj, 0, st_);
            k_cgs(ka, jj, 1, st_);
            k_cgs(ka, jj, 2, st_);
            k_normalize(ka, jj, last_allowed, st_);
        };
        // every step of this cycle in one persistent launch (the default for
        // precisions 0 and 1 when the profile is off)
        const bool use_persist = S.persist_ok && !persist_off && !nested && !S.prof && ka.grp <= 1;
        if (use_persist) {
            if (!S.d_pbar) {
                S.d_pbar = S.dalloc<unsigned int>(1, S.allocs);
                S.d_pstatus = S.dalloc<int>(1, S.allocs);
            }
            PersistArgs pa;
            std::memset(&pa, 0, sizeof(pa));
            pa.ka = ka;
            GemmCall calls[2];
            for (int set = 0; set < 2; ++set) {
                if (set == 1 && !bj_fp32) break;
                pa.nbj[set] = bj_calls(S, w.V, (long long)(m + 1) * ld, 0, w.z, ld, 0, w.active, set == 1, calls);
                for (int i = 0; i < pa.nbj[set]; ++i) pa.bj[set][i] = to_pgemm(S, calls[i]);
            }
            pa.nsc = schur_calls(S, w.z, ld, 0, w.w, w.z, w.active, false, calls);
            for (int i = 0; i < pa.nsc; ++i) pa.sc[i] = to_pgemm(S, calls[i]);
            pa.bj_step = ld;
            pa.j0 = 0;
            pa.last_allowed = last_allowed;
            pa.use_fp32 = bj_fp32 ? 1 : 0;
            pa.fp64_steps = cycles == 0 ? check_every : 0;    // precision 1: the first group in FP64
            pa.Zb = mixed ? w.Zb : nullptr;
            pa.z = w.z;
            pa.bar = S.d_pbar;
            pa.status = S.d_pstatus;
            pa.wait_ns = persist_wait_ns;
            pa.stall = persist_stall ? 1 : 0;
            CK(cudaMemsetAsync(S.d_pbar, 0, sizeof(unsigned int), st_));
            CK(cudaMemsetAsync(S.d_pstatus, 0, sizeof(int), st_));
            if (k_arnoldi_persistent(pa, st_)) {
                int h_status = 0;
                CK(cudaMemcpyAsync(&h_status, S.d_pstatus, sizeof(int), cudaMemcpyDeviceToHost, st_));
                CK(cudaMemcpyAsync(h_active.data(), w.active, R * sizeof(int), cudaMemcpyDeviceToHost, st_));
                CK(cudaStreamSynchronize(st_));
                if (h_status != 0)
                    throw Err{SMPM_ETIMEOUT, "persistent Arnoldi kernel: a grid barrier wait ran out of time"};
                j = last_allowed;
            } else {
                cudaGetLastError();
                S.persist_ok = false;                   // step-group launches from now on
            }
        }
        while (j < last_allowed) {
            const int cnt = std::min(check_every - j % check_every, last_allowed - j);
            // precision 1: the first step group of the first cycle applies the
            // FP64 blocks (easy problems -- large k^2 -- converge right there,
            // where FP32 copies of their ill-conditioned blocks would stall the
            // flexible GMRES near 1e-8); FP32 from the next group on
            group_fp32 = bj_fp32 && !(cycles == 0 && j < check_every);
            const std::array<int, 4> key{j, cnt, last_allowed, group_fp32 ? 1 : 0};
            Solver::GroupGraph* gg = nullptr;
            if (use_graphs) {
                auto it = S.graphs.find(key);
                if (it != S.graphs.end()) {
                    gg = &it->second;
                } else if (++S.group_seen[key] >= 2) {
                    // capture the group on a side stream, launch it on the solver's
                    if (!S.cap_stream) CK(cudaStreamCreateWithFlags(&S.cap_stream, cudaStreamNonBlocking));
                    Solver::GroupGraph g_new;
                    cudaStream_t keep = S.stream;
                    S.stream = st_ = S.cap_stream;
                    if (S.prof) {
                        S.cap_events = &g_new.ev;
                        S.cap_f32 = &g_new.f32;
                    }
                    const long long l0 = launch_count();
                    cudaGraph_t graph = nullptr;
                    cudaError_t e1 = cudaStreamBeginCapture(S.cap_stream, cudaStreamCaptureModeThreadLocal);
                    if (e1 == cudaSuccess) {
                        S.capturing = true;
                        try {
                            for (int jj = j; jj < j + cnt; ++jj) step(jj);
                        } catch (...) {
                            cudaStreamEndCapture(S.cap_stream, &graph);
                            if (graph) cudaGraphDestroy(graph);
                            S.stream = st_ = keep;
                            S.cap_events = nullptr;
                            S.cap_f32 = nullptr;
                            S.capturing = false;
                            throw;
                        }
                        S.capturing = false;
                        e1 = cudaStreamEndCapture(S.cap_stream, &graph);
                    }
                    S.stream = st_ = keep;
                    S.cap_events = nullptr;
                    S.cap_f32 = nullptr;
                    g_new.launches = launch_count() - l0;
                    count_launches((int)-g_new.launches);     // counted again at every replay
                    if (e1 == cudaSuccess && graph)
                        e1 = cudaGraphInstantiate(&g_new.exec, graph, 0);
                    if (graph) cudaGraphDestroy(graph);
                    if (e1 != cudaSuccess || !g_new.exec) {
                        cudaGetLastError();
                        for (cudaEvent_t e : g_new.ev) cudaEventDestroy(e);
                        S.graphs_ok = false;                 // direct launches from now on
                    } else {
                        gg = &(S.graphs[key] = std::move(g_new));
                    }
                }
            }
            if (gg) {
                CK(cudaGraphLaunch(gg->exec, st_));
                count_launches((int)gg->launches);
            } else {
                for (int jj = j; jj < j + cnt; ++jj) step(jj);
            }
            j += cnt;
            CK(cudaMemcpyAsync(h_active.data(), w.active, R * sizeof(int), cudaMemcpyDeviceToHost, st_));
            CK(cudaStreamSynchronize(st_));
            if (gg && S.prof) {
                for (size_t e = 0; e + 1 < gg->ev.size(); e += 2) {
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, gg->ev[e], gg->ev[e + 1]));
                    add_prof(S, gg->f32[e / 2], 1, ms, 0.0);
                }
            }
            bool any = false;
            for (int r = 0; r < R; ++r) any |= h_active[r] != 0;
            if (!any) break;
        }
        CK(cudaMemcpyAsync(h_nit.data(), w.nit, R * sizeof(int), cudaMemcpyDeviceToHost, st_));
        if (mixed) {
            k_cycle_update(ka, w.t, st_, w.Zb, (long long)m * ld);  // t = sum y_j z_j (FGMRES)
        } else {
            k_cycle_update(ka, w.Xp, st_);             // Y = V y
            bj(w.Xp, ld, 0, w.t, ld, 0, nullptr);      // t = M^-1 Y
        }
        schur(w.t, ld, 0, w.s, nullptr);               // S t
        k_deflate_coarse_pending(ka, w.s, st_);        // c = K Z^T S t
        k_xs_update(ka, w.xS, w.t, w.c0, st_);         // x_S += t + Z (c0 - c)
        // k^2 = 0: drop the component of x_S along the right null vector 1_S
        // (S 1_S = 0, so S x_S is unchanged).  Left in place it grows from
        // cycle to cycle and sets a rounding floor e |G| |x_S| on the true
        // residual (seen as stagnation near 2e-10 on 512 x 16, order 12).
        k_dot_partial(R, S.kp, w.xS, ld, w.oneSp, w.rpart, nch, kChunk, st_);
        k_project(R, S.kp, w.xS, ld, w.oneSp, w.rpart, nch, kChunk, st_);
        CK(cudaStreamSynchronize(st_));
        int mx_it = 0;
        for (int r = 0; r < R; ++r) mx_it = std::max(mx_it, h_nit[r]);
        for (int r = 0; r < R; ++r) h_base[r] = std::min(h_base[r] + h_nit[r], S.max_iter);
        total_it += std::max(mx_it, 1);
        ++cycles;
        first = false;
    }
    S.hist_steps = h_base;
    S.hist_R = R;
    phase("cycles");
    // recovery: u = A^-1 (b - E x_S)  (Alg. seq step 9)
    if (S.fss) {
        fss_refined(S, fa, R, w.b, g.r, u_d, g.r, w.xS, ld, w.k2r, w.fs1, w.fs2, w.fs3, w.tS1, w.tS2);
    } else {
        k_recovery_rhs(ga, R, w.b, g.r, w.xS, ld, w.t2, st_);
        GemmArgs a = gemm_base(S);
        a.mats = S.Ainv; a.mat_stride = S.sA; a.M = nfz; a.K = nfz;
        a.row_lo = S.rl_A; a.row_hi = S.rh_A;
        a.in = w.t2; a.in_rs = g.r; a.in_us = nfz; a.in_off = 0;
        a.out = u_d; a.out_rs = g.r; a.out_us = nfz; a.out_off0 = 0; a.out_off1 = 0; a.msplit = nfz;
        run_gemm(S, a, w.tA, 0);
    }
    k_gauge(ga, R, u_d, g.r, w.gauge, w.rpart, rch, kChunk, st_);
    phase("recovery");
    if (tphase) fprintf(stderr, "smpm solve phases (ms, R=%d, %d cycles):%s\n", R, cycles, tp_msg.c_str());
    if (!u_dev) CK(cudaMemcpyAsync(u, u_d, sizeof(double) * g.r * R, cudaMemcpyDeviceToHost, st_));
    std::vector<double> h_r(R), h_b(R);
    CK(cudaMemcpyAsync(h_r.data(), w.rnorm, R * sizeof(double), cudaMemcpyDeviceToHost, st_));
    CK(cudaMemcpyAsync(h_b.data(), w.bnorm, R * sizeof(double), cudaMemcpyDeviceToHost, st_));
    CK(cudaMemcpyAsync(h_flags.data(), w.flags, R * sizeof(int), cudaMemcpyDeviceToHost, st_));
    int h_ozerr = 0;
    if (S.d_ozerr) CK(cudaMemcpyAsync(&h_ozerr, S.d_ozerr, sizeof(int), cudaMemcpyDeviceToHost, st_));
    CK(cudaStreamSynchronize(st_));
    if (h_ozerr != 0) {
        CK(cudaMemsetAsync(S.d_ozerr, 0, sizeof(int), st_));
        throw Err{SMPM_ETIMEOUT, "tensor-core product: a wait for a copy or the tensor pipe ran out of iterations"};
    }
    CK(cudaGetLastError());
    harvest_profile(S);
    double worst = 0.0;
    if (stagnated && status == SMPM_OK) status = SMPM_ENOCONV;
    for (int r = 0; r < R; ++r) {
        const double rel = h_b[r] > 0 ? h_r[r] / h_b[r] : 0.0;
        worst = std::max(worst, rel);
        if (h_flags[r] & 1) status = SMPM_EBREAKDOWN;
        if (!std::isfinite(rel)) status = SMPM_EBREAKDOWN;
    }
    S.last_res.assign(R, 0.0);
    for (int r = 0; r < R; ++r) S.last_res[r] = h_b[r] > 0 ? h_r[r] / h_b[r] : 0.0;
    if (st) {
        st->iters = total_it;
        st->restarts = std::max(0, cycles - 1);
        st->status = status;
        st->rel_resid_true = worst;
        st->setup_ms = S.setup_ms;
        st->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

// One operator of the method applied to nrhs vectors (parity checks of the
// individual kernels): kind 0: S x (Sec. 2.3); 1: M^-1 x (Sec. 3.2);
// 2: P x = x - S Z K Z^T x (Sec. 3.3); 3: b_S = B A^-1 b (r -> k);
// 4: A^-1 b per strip (r -> r).  Face vectors use the unpadded interface order
// (2 j + s) fz + Z of length k.
static int apply_impl(Solver& S, int kind, int R, const double* in, double* out) {
    if (R <= 0 || !in || !out) throw Err{SMPM_EINVAL, "bad apply arguments"};
    if (kind < 0 || kind > 4) throw Err{SMPM_EINVAL, "unknown operator kind"};
    std::vector<int> ops(R, 0);
    ensure_workspace(S, R);
    prepare_ops(S, ops);
    const Geometry& g = S.g;
    auto& w = S.wk;
    cudaStream_t st_ = S.stream;
    const int fz = g.fz, nfz = g.n * fz, f2 = 2 * fz, f4 = 4 * fz;
    const long long ld = S.ld, k = g.k, r = g.r;
    const bool face_in = kind <= 2, face_out = kind <= 3;
    const cudaMemcpyKind kin = is_device_ptr(in) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (face_in)
        CK(cudaMemcpy2DAsync(w.z + fz, ld * 8, in, k * 8, k * 8, R, kin, st_));
    else
        CK(cudaMemcpyAsync(w.t2, in, sizeof(double) * r * R, kin, st_));
    std::vector<int> ones(R, 1);
    CK(cudaMemcpyAsync(w.active, ones.data(), R * sizeof(int), cudaMemcpyHostToDevice, st_));
    double* res = w.w;
    GemmArgs a;
    std::memset(&a, 0, sizeof(a));
    if (kind == 0) {
        schur_product(S, w.z, ld, 0, w.w, w.z, nullptr, false);
    } else if (kind == 1) {
        // precision 2 keeps only the FP32 block inverses
        bj_apply(S, w.z, ld, 0, w.w, ld, 0, nullptr, S.precision == 2);
    } else if (kind == 2) {
        KArgs ka;
        std::memset(&ka, 0, sizeof(ka));
        const int m = S.restart;
        ka.R = R; ka.m = m; ka.nch = (int)((S.kp + kChunk - 1) / kChunk); ka.ch = kChunk; ka.ld = ld; ka.kp = S.kp;
        ka.fz = fz; ka.mx = g.mx; ka.ng = g.ng; ka.d = g.d; ka.n = g.n;
        ka.V = w.V; ka.w = w.w; ka.Hc = w.Hc; ka.htmp = w.htmp; ka.cs = w.cs; ka.sn = w.sn; ka.gv = w.gv;
        ka.part1 = w.part1; ka.part2 = w.part2; ka.q = w.q; ka.c = w.c;
        ka.rho = S.rho; ka.rho_stride = S.sRho; ka.K = S.K; ka.K_stride = S.sK;
        ka.op = w.op; ka.strip_cls = S.d_strip_cls;
        ka.active = w.active; ka.done = w.done; ka.nit = w.nit; ka.target = w.target;
        ka.bnorm = w.bnorm; ka.rnorm = w.rnorm; ka.flags = w.flags;
        CK(cudaMemcpyAsync(w.w, w.z, sizeof(double) * ld * R, cudaMemcpyDeviceToDevice, st_));
        k_deflate_sum(ka, w.w, nullptr, st_);
        k_coarse(ka, st_);
        k_cgs(ka, -1, 0, st_);  // w -= S Z c, no dot products
    } else if (kind == 3 && S.fss) {
        const FssArgs fa{g.n, fz, g.mx, S.d_strip_cls};
        fss_refined(S, fa, R, w.t2, r, w.b, r, nullptr, 0, w.k2r, w.fs1, w.fs2, w.fs3, w.tS1, w.tS2);
        k_face_flux(fa, R, S.d_beta, w.b, r, w.w, ld, S.kp, st_);
    } else if (kind == 4 && S.fss) {
        const FssArgs fa{g.n, fz, g.mx, S.d_strip_cls};
        fss_refined(S, fa, R, w.t2, r, w.b, r, nullptr, 0, w.k2r, w.fs1, w.fs2, w.fs3, w.tS1, w.tS2);
        res = w.b;
    } else if (kind == 3) {
        a.mats = S.W; a.mat_stride = S.sW; a.M = f2; a.K = nfz; a.row_lo = S.rl_GW; a.row_hi = S.rh_GW;
        a.in = w.t2; a.in_rs = r; a.in_us = nfz; a.in_off = 0;
        a.out = w.w; a.out_rs = ld; a.out_us = f2; a.out_off0 = -fz; a.out_off1 = f2; a.msplit = fz;
        run_gemm(S, a, w.tW, 0);
    } else {
        a.mats = S.Ainv; a.mat_stride = S.sA; a.M = nfz; a.K = nfz; a.row_lo = S.rl_A; a.row_hi = S.rh_A;
        a.in = w.t2; a.in_rs = r; a.in_us = nfz; a.in_off = 0;
        a.out = w.b; a.out_rs = r; a.out_us = nfz; a.msplit = nfz;
        run_gemm(S, a, w.tA, 0);
        res = w.b;
    }
    if (face_out)
        CK(cudaMemcpy2DAsync(out, k * 8, res + fz, ld * 8, k * 8, R, kout, st_));
    else
        CK(cudaMemcpyAsync(out, res, sizeof(double) * r * R, kout, st_));
    CK(cudaStreamSynchronize(st_));
    CK(cudaGetLastError());
    harvest_profile(S);
    return SMPM_OK;
}

static void profile_enable(Solver& S, bool enable) {
    if (enable && S.ev.empty()) {
        S.ev.resize(2 * kEventPairs);
        S.ev_f32.assign(kEventPairs, 0);
        for (auto& e : S.ev) CK(cudaEventCreate(&e));
        S.d_flops = S.dalloc<unsigned long long>(4, S.allocs);
        CK(cudaMemsetAsync(S.d_flops, 0, 4 * sizeof(unsigned long long), S.stream));
    }
    if (S.prof != enable) {
        CK(cudaStreamSynchronize(S.stream));
        S.drop_graphs();
    }
    S.prof = enable;
}

// Totals of precision p (0 FP64, 1 FP32) of handle h, or of the process for h = NULL.
static void read_prof(smpm_handle h, int p, int reset, long long& n, double& f, double& t) {
    if (h) {
        Solver& S = *(Solver*)h;
        n += S.prof_launches[p];
        f += S.prof_flops[p];
        t += S.prof_ms[p];
        if (reset) { S.prof_launches[p] = 0; S.prof_flops[p] = 0.0; S.prof_ms[p] = 0.0; }
        return;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    n += g_prof_launches[p];
    f += g_prof_flops[p];
    t += g_prof_ms[p];
    if (reset) { g_prof_launches[p] = 0; g_prof_flops[p] = 0.0; g_prof_ms[p] = 0.0; }
}

static Solver* make_solver(const smpm_grid* grid, int nop, const double* k2, void* stream) {
    if (!grid) throw Err{SMPM_EINVAL, "grid is null"};
    if (nop < 1) throw Err{SMPM_EINVAL, "need at least one k^2"};
    auto S = std::make_unique<Solver>();
    S->opt = *grid;
    std::string msg;
    if (!make_geometry(grid->mx, grid->mz, grid->order, grid->lx, grid->lz, grid->z_ratio, grid->tau_scale,
                       grid->deflation_groups, S->g, msg))
        throw Err{SMPM_EINVAL, msg};
    if (grid->precision < 0 || grid->precision > 2)
        throw Err{SMPM_EINVAL, "precision must be 0 (FP64), 1 (FP32 block-Jacobi) or 2 (FP32 inner DBJ-GMRES)"};
    if (grid->krylov < 0 || grid->krylov > 1)
        throw Err{SMPM_EINVAL, "krylov must be 0 (one Krylov space per right-hand side) or 1 (concatenated)"};
    S->nop = nop;
    S->k2.assign(k2, k2 + nop);
    int nzero = 0;
    for (double v : S->k2) {
        if (!(v >= 0.0) || !std::isfinite(v)) throw Err{SMPM_EINVAL, "k2 must be finite and >= 0"};
        if (v == 0.0) ++nzero;
    }
    if (nzero > 1) throw Err{SMPM_EINVAL, "at most one k2 = 0 operator per handle"};
    S->stream = (cudaStream_t)stream;
    S->precision = grid->precision;
    S->krylov = grid->krylov;
    if (const char* e = std::getenv("SMPM_INNER_STEPS"))   // inner Arnoldi steps of precision 2
        S->inner_m = std::min(64, std::max(2, std::atoi(e)));
    setup_solver(*S);
    if (g_prof_default.load()) profile_enable(*S, true);
    return S.release();
}

template <class F>
static int guarded(F&& fn) {
    try {
        g_last_error.clear();
        return fn();
    } catch (const Err& e) {
        g_last_error = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return SMPM_ECUDA;
    } catch (...) {
        g_last_error = "unknown error";
        return SMPM_ECUDA;
    }
}

// Operator data of operator set 0 for the allocation-free deflation
// projection (noalloc.cu); reads the handle only.

bool deflation_view(smpm_handle h, DeflView* v, std::string& msg) {
    if (!h) { msg = "null handle"; return false; }
    const Solver& S = *(const Solver*)h;
    v->fz = S.g.fz; v->mx = S.g.mx; v->ng = S.g.ng; v->d = S.g.d; v->k = S.g.k;
    v->K = S.K; v->rho = S.rho; v->strip_cls = S.d_strip_cls; v->stream = S.stream;
    return true;
}

void set_last_error(const std::string& msg) { g_last_error = msg; }

}  // namespace smpm

using namespace smpm;

extern "C" {

int smpm_setup(const smpm_grid* grid, double k2, void* stream, smpm_handle* out) {
    return guarded([&] {
        if (!out) throw Err{SMPM_EINVAL, "out is null"};
        *out = (smpm_handle)make_solver(grid, 1, &k2, stream);
        return SMPM_OK;
    });
}

int smpm_solve_guess(smpm_handle h, int nrhs, const double* f, const double* g, const double* u0, double tol,
                     double* u, smpm_stats* st) {
    return guarded([&] {
        if (!h) throw Err{SMPM_EINVAL, "null handle"};
        if (nrhs <= 0) throw Err{SMPM_EINVAL, "nrhs must be positive"};
        Solver& S = *(Solver*)h;
        std::vector<int> ops((size_t)nrhs, 0);
        return solve_impl(S, ops, f, g, tol, u, st, u0);
    });
}

int smpm_setup_multi(const smpm_grid* grid, int nop, const double* k2, void* stream, smpm_handle* out) {
    return guarded([&] {
        if (!out || !k2) throw Err{SMPM_EINVAL, "null argument"};
        *out = (smpm_handle)make_solver(grid, nop, k2, stream);
        return SMPM_OK;
    });
}

int smpm_solve(smpm_handle h, const double* f, const double* g, double tol, double* u, smpm_stats* st) {
    return guarded([&] {
        if (!h) throw Err{SMPM_EINVAL, "null handle"};
        std::vector<int> ops(1, 0);
        return solve_impl(*(Solver*)h, ops, f, g, tol, u, st);
    });
}

int smpm_solve_batch(smpm_handle h, int nrhs, const double* f, const double* g, double tol, double* u,
                     smpm_stats* st) {
    return guarded([&] {
        if (!h) throw Err{SMPM_EINVAL, "null handle"};
        if (nrhs <= 0) throw Err{SMPM_EINVAL, "nrhs must be positive"};
        std::vector<int> ops(nrhs, 0);
        return solve_impl(*(Solver*)h, ops, f, g, tol, u, st);
    });
}

int smpm_solve_multi(smpm_handle h, int nrhs, const int* op_of_rhs, const double* f, const double* g, double tol,
                     double* u, smpm_stats* st) {
    return guarded([&] {
        if (!h || !op_of_rhs) throw Err{SMPM_EINVAL, "null argument"};
        Solver& S = *(Solver*)h;
        if (nrhs <= 0) throw Err{SMPM_EINVAL, "nrhs must be positive"};
        std::vector<int> ops(op_of_rhs, op_of_rhs + nrhs);
        for (int o : ops)
            if (o < 0 || o >= S.nop) throw Err{SMPM_EINVAL, "operator index out of range"};
        for (int r = 1; r < nrhs; ++r)
            if (ops[r] < ops[r - 1]) throw Err{SMPM_EINVAL, "op_of_rhs must be non-decreasing"};
        return solve_impl(S, ops, f, g, tol, u, st);
    });
}

int smpm_apply(smpm_handle h, int kind, int nrhs, const double* in, double* out) {
    return guarded([&] {
        if (!h) throw Err{SMPM_EINVAL, "null handle"};
        return apply_impl(*(Solver*)h, kind, nrhs, in, out);
    });
}

int smpm_setup_3d(const smpm_grid* grid, int my, double ly, void* stream, smpm_handle* out) {
    return guarded([&] {
        if (!out) throw Err{SMPM_EINVAL, "out is null"};
        if (my < 2 || my % 2 != 0) throw Err{SMPM_EINVAL, "my must be even and >= 2"};
        if (!(ly > 0.0)) throw Err{SMPM_EINVAL, "ly must be positive"};
        const int nm = my / 2 + 1;
        std::vector<double> k2(nm);
        const double pi = 3.14159265358979323846;
        for (int j = 0; j < nm; ++j) {
            const double kj = 2.0 * pi * j / ly;
            k2[j] = kj * kj;
        }
        Solver* S = make_solver(grid, nm, k2.data(), stream);
        S->my = my;
        *out = (smpm_handle)S;
        return SMPM_OK;
    });
}

int smpm_solve_3d_physical(smpm_handle h, const double* f3, const double* g3, double tol, double* u3,
                           smpm_stats* st) {
    return guarded([&] {
        if (!h || !f3 || !u3) throw Err{SMPM_EINVAL, "null argument"};
        Solver& S = *(Solver*)h;
        if (S.my <= 0) throw Err{SMPM_EINVAL, "the handle was not built by smpm_setup_3d"};
        const auto t0 = std::chrono::steady_clock::now();
        const int my = S.my, nm = my / 2 + 1;
        const long long r = S.g.r, nb = 2LL * S.g.fz + 2LL * S.g.nx;
        cudaStream_t st_ = S.stream;
        if (!S.d_cs) {
            // exact zeros and ones at the quarter points keep mode 0 and the
            // Nyquist mode real
            std::vector<double> cs(2 * (size_t)my);
            const long double pi = 3.141592653589793238462643383279502884L;
            for (int i = 0; i < my; ++i) {
                const long double a = 2.0L * pi * i / my;
                cs[i] = (4 * i == my || 4 * i == 3 * my) ? 0.0 : (double)std::cos(a);
                cs[my + i] = (i == 0 || 2 * i == my) ? 0.0 : (double)std::sin(a);
            }
            S.d_cs = S.dalloc<double>(cs.size(), S.allocs);
            upload(S.d_cs, cs, st_);
        }
        if (S.cap3 < r) {
            S.f3hat = S.dalloc<double>((size_t)nm * 2 * r, S.allocs);
            S.u3hat = S.dalloc<double>((size_t)nm * 2 * r, S.allocs);
            S.f3stage = S.dalloc<double>((size_t)my * r, S.allocs);
            S.cap3 = r;
        }
        if (g3 && S.capg3 < nb) {
            S.g3hat = S.dalloc<double>((size_t)nm * 2 * nb + (size_t)my * nb, S.allocs);
            S.capg3 = nb;
        }
        const double* f_d = f3;
        if (!is_device_ptr(f3)) {
            CK(cudaMemcpyAsync(S.f3stage, f3, sizeof(double) * my * r, cudaMemcpyHostToDevice, st_));
            f_d = S.f3stage;
        }
        k_dft_forward(f_d, S.f3hat, S.d_cs, r, my, st_);
        double* gh = nullptr;
        if (g3) {
            gh = S.g3hat;
            const double* g_d = g3;
            if (!is_device_ptr(g3)) {
                double* gstage = S.g3hat + (size_t)nm * 2 * nb;
                CK(cudaMemcpyAsync(gstage, g3, sizeof(double) * my * nb, cudaMemcpyHostToDevice, st_));
                g_d = gstage;
            }
            k_dft_forward(g_d, gh, S.d_cs, nb, my, st_);
        }
        std::vector<int> ops(2 * S.nop);
        for (int j = 0; j < S.nop; ++j) ops[2 * j] = ops[2 * j + 1] = j;
        const int rc = solve_impl(S, ops, S.f3hat, gh, tol, S.u3hat, st);
        double* u_d = is_device_ptr(u3) ? u3 : S.f3stage;
        k_dft_inverse(S.u3hat, u_d, S.d_cs, r, my, st_);
        if (u_d != u3) CK(cudaMemcpyAsync(u3, u_d, sizeof(double) * my * r, cudaMemcpyDeviceToHost, st_));
        CK(cudaStreamSynchronize(st_));
        if (st) st->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        return rc;
    });
}

int smpm_solve_3d(smpm_handle h, const double* fhat, const double* ghat, double tol, double* uhat,
                  smpm_stats* st) {
    return guarded([&] {
        if (!h) throw Err{SMPM_EINVAL, "null handle"};
        Solver& S = *(Solver*)h;
        std::vector<int> ops(2 * S.nop);
        for (int j = 0; j < S.nop; ++j) ops[2 * j] = ops[2 * j + 1] = j;
        return solve_impl(S, ops, fhat, ghat, tol, uhat, st);
    });
}

int smpm_sizes(smpm_handle h, long long* r, long long* nb, long long* k) {
    return guarded([&] {
        if (!h) throw Err{SMPM_EINVAL, "null handle"};
        const Solver& S = *(Solver*)h;
        if (r) *r = S.g.r;
        if (nb) *nb = 2LL * S.g.fz + 2LL * S.g.nx;
        if (k) *k = S.g.k;
        return SMPM_OK;
    });
}

static void fill_coords(const Geometry& g, double* x, double* z) {
    for (int X = 0; X < g.nx; ++X) {
        const int ex = X / g.n, a = X % g.n;
        const double xv = ex * g.hx + (g.xi[a] + 1.0) * g.hx * 0.5;
        for (int Z = 0; Z < g.fz; ++Z) {
            const int ez = Z / g.n, b = Z % g.n;
            x[(size_t)X * g.fz + Z] = xv;
            z[(size_t)X * g.fz + Z] = g.zb[ez] + (g.xi[b] + 1.0) * g.hz[ez] * 0.5;
        }
    }
}

int smpm_node_coords(smpm_handle h, double* x, double* z) {
    return guarded([&] {
        if (!h || !x || !z) throw Err{SMPM_EINVAL, "null argument"};
        fill_coords(((Solver*)h)->g, x, z);
        return SMPM_OK;
    });
}

int smpm_grid_coords(const smpm_grid* grid, double* x, double* z) {
    return guarded([&] {
        if (!grid || !x || !z) throw Err{SMPM_EINVAL, "null argument"};
        Geometry g;
        std::string msg;
        if (!make_geometry(grid->mx, grid->mz, grid->order, grid->lx, grid->lz, grid->z_ratio, grid->tau_scale,
                           grid->deflation_groups, g, msg))
            throw Err{SMPM_EINVAL, msg};
        fill_coords(g, x, z);
        return SMPM_OK;
    });
}

int smpm_last_residuals(smpm_handle h, int n, double* out) {
    return guarded([&] {
        if (!h || !out) throw Err{SMPM_EINVAL, "null argument"};
        const Solver& S = *(Solver*)h;
        if (n > (int)S.last_res.size()) throw Err{SMPM_EINVAL, "more values requested than the last solve had"};
        for (int i = 0; i < n; ++i) out[i] = S.last_res[i];
        return SMPM_OK;
    });
}

int smpm_residual_history(smpm_handle h, int rhs, int kind, int n, double* out, int* count) {
    return guarded([&] {
        if (!h || !count) throw Err{SMPM_EINVAL, "null argument"};
        Solver& S = *(Solver*)h;
        if (rhs < 0 || rhs >= S.hist_R) throw Err{SMPM_EINVAL, "rhs out of range of the last solve"};
        if (kind != 0 && kind != 1) throw Err{SMPM_EINVAL, "kind must be 0 (per Arnoldi step) or 1 (per cycle)"};
        if (n < 0 || (n > 0 && !out)) throw Err{SMPM_EINVAL, "n must be >= 0 and out non-null when n > 0"};
        if (kind == 1) {
            const auto& v = S.hist_true[rhs];
            *count = (int)v.size();
            std::copy(v.begin(), v.begin() + std::min<size_t>(n, v.size()), out);
            return SMPM_OK;
        }
        const int steps = S.hist_steps[rhs];
        *count = steps;
        const int k = std::min(n, steps);
        if (k > 0) {
            CK(cudaMemcpyAsync(out, S.wk.hist + (size_t)rhs * (S.max_iter + 1) + 1, sizeof(double) * k,
                               cudaMemcpyDeviceToHost, S.stream));
            CK(cudaStreamSynchronize(S.stream));
        }
        return SMPM_OK;
    });
}

int smpm_null_vectors(smpm_handle h, double* uL, double* uS) {
    return guarded([&] {
        if (!h || !uL || !uS) throw Err{SMPM_EINVAL, "null argument"};
        const Solver& S = *(Solver*)h;
        if (S.singular_op < 0) throw Err{SMPM_EINVAL, "the handle has no k^2 = 0 operator set"};
        const cudaMemcpyKind kl = is_device_ptr(uL) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        const cudaMemcpyKind ks = is_device_ptr(uS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(uL, S.uL, sizeof(double) * S.g.r, kl, S.stream));
        CK(cudaMemcpyAsync(uS, S.uS + S.g.fz, sizeof(double) * S.g.k, ks, S.stream));
        CK(cudaStreamSynchronize(S.stream));
        return SMPM_OK;
    });
}

int smpm_set_stream(smpm_handle h, void* stream) {
    return guarded([&] {
        if (!h) throw Err{SMPM_EINVAL, "null handle"};
        Solver& S = *(Solver*)h;
        if (S.stream) CK(cudaStreamSynchronize(S.stream));
        S.stream = (cudaStream_t)stream;
        return SMPM_OK;
    });
}

long long smpm_device_bytes(smpm_handle h) { return h ? ((Solver*)h)->bytes : 0; }

void smpm_release(smpm_handle h) {
    try {
        delete (Solver*)h;
    } catch (...) {
    }
}

const char* smpm_last_error(void) { return g_last_error.c_str(); }

int smpm_profile(smpm_handle h, int enable) {
    return guarded([&] {
        if (!h) {   // process-wide default for the handles created from now on
            g_prof_default.store(enable != 0);
            return SMPM_OK;
        }
        profile_enable(*(Solver*)h, enable != 0);
        return SMPM_OK;
    });
}

int smpm_profile_read(smpm_handle h, long long* launches, double* flops, double* ms, int reset) {
    return guarded([&] {
        long long n = 0;
        double f = 0.0, t = 0.0;
        for (int p = 0; p < 3; ++p) read_prof(h, p, reset, n, f, t);
        if (reset) {
            long long n3 = 0;
            double f3 = 0.0, t3 = 0.0;
            read_prof(h, 3, reset, n3, f3, t3);
        }
        if (launches) *launches = n;
        if (flops) *flops = f;
        if (ms) *ms = t;
        return SMPM_OK;
    });
}

int smpm_profile_split(smpm_handle h, int precision, long long* launches, double* flops, double* ms, int reset) {
    return guarded([&] {
        if (precision < 0 || precision > 3)
            throw Err{SMPM_EINVAL, "category must be 0 (FP64), 1 (FP32), 2 (tensor, algorithmic) or 3 (tensor, executed)"};
        long long n = 0;
        double f = 0.0, t = 0.0;
        read_prof(h, precision, reset, n, f, t);
        if (launches) *launches = n;
        if (flops) *flops = f;
        if (ms) *ms = t;
        return SMPM_OK;
    });
}

long long smpm_kernel_launches(void) { return launch_count(); }

int smpm_probe_fp64(void* stream, double* tflops) {
    return guarded([&] {
        if (!tflops) throw Err{SMPM_EINVAL, "null argument"};
        cudaStream_t s = (cudaStream_t)stream;
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        double* out = nullptr;
        CK(cudaMalloc(&out, sizeof(double) * 4096));
        const int blocks = sms * 8, iters = 4096;
        k_fp64_probe(out, blocks, 64, s);
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, s));
        k_fp64_probe(out, blocks, iters, s);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(out);
        const double flops = 2.0 * 8.0 * 256.0 * (double)blocks * (double)iters;
        *tflops = flops / (ms * 1e-3) / 1e12;
        return SMPM_OK;
    });
}

}  // extern "C"

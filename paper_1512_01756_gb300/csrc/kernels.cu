// Device kernels of libsmpm (FP64, sm_103a).
//
// Hot path of Alg. seq (Sec. 3): the Schur product S x = x + sum_i scatter_i(G_i gather_i x)
// (Sec. 2.3 / 3.1, assembled form), the block-Jacobi apply M^-1 (Sec. 3.2), the
// deflation Z^T, coarse solve and S Z c correction (Sec. 3.3), classical
// Gram-Schmidt applied twice with Givens rotations (Arnoldi of GMRES), the
// null-space projections (Eqs. regularize_poisson / regularize_schur) and the
// strip solves A^-1 of the right-hand side and of the recovery step.
//
// FP64 arithmetic is bound by the DFMA pipe on this part, so the dense applies
// are register-tiled SIMT GEMMs over tiles that share one class matrix; the
// vector kernels are chunked streams over the face vectors.
#include <mutex>
#include <algorithm>
#include <atomic>
#include <cmath>

#include "kernels.h"

namespace smpm {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launches(int n) { g_launches.fetch_add(n); }

#define CUDA_LAUNCH_CHECK() (void)0

static constexpr int BM = 16, BK = 16, GT = 128;   // default tile rows, K slab, threads per GEMM CTA
static constexpr int VB = 256;  // threads of the vector kernels

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over a block of NT threads; every thread gets the result.
template <int NT = VB>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = lane < (NT / 32) ? sh[lane] : 0.0;
    t = warp_sum(t);
    return t;
}

// ---------------------------------------------------------------------------
// Class GEMM: out[:, col] = Mat_{tile} * in[:, col] (+ add) over tiles of columns
// sharing one class matrix.  A CTA of 128 threads owns a BMT-row x BNT-column
// output tile, each thread one row and four columns: 16 x 32 (the default) or
// 8 x 64 (less row padding for small M such as the f_z-row slot matrices).
// The short row tiles keep the padding waste of M = f_z, 2 f_z, 4 f_z small,
// and the many small tiles spread the FP64 work evenly over the SMs.  K runs
// in 16-wide slabs; the last slab stops at K (no FMAs on padding).
// ---------------------------------------------------------------------------
// TM: element type of the class matrices and of the arithmetic (double, or
// float for the FP32 block-Jacobi of the mixed-precision solve: FP64 vectors are
// rounded to FP32 on load, products accumulate in FP32, results are stored in FP64).
// Shared-memory words of one GEMM tile: the A slab (BK x (BMT + 1)) and the
// B slab (BK x (BNT + 4)), both a multiple of 16 bytes; twice that for the
// mirror form (two A and two B slabs).
template <typename TM, int BMT>
__host__ __device__ constexpr int gemm_smem_words() {
    return BK * (BMT + 1) + BK * (4 * GT / BMT + 4);
}

// One BMT x BNT output tile of the class GEMM: tile t of the launch, row tile
// `by`; As_ / Bs_ are the tile's shared slabs (16-byte aligned).  Run by GT
// threads (threadIdx.x < GT) of one block.
template <int EPI, typename TM, int BMT>
__device__ __forceinline__ void class_gemm_tile(const GemmArgs& a, const Tile t, int by, TM* As_, TM* Bs_) {
    constexpr int BNT = 4 * GT / BMT;          // columns per tile (4 per thread)
    constexpr int CG = GT / BMT;               // column groups of four
    auto As = reinterpret_cast<TM (*)[BMT + 1]>(As_);
    auto Bs = reinterpret_cast<TM (*)[BNT + 4]>(__builtin_assume_aligned(Bs_, 16));
    const int row0 = by * BMT;
    const int lo = a.row_lo[t.mat], hi = a.row_hi[t.mat];
    if (row0 >= hi || row0 + BMT <= lo) return;
    if (a.active) {
        int any = 0;
        for (int c = 0; c < t.nr; ++c) any |= a.active[t.r0 + c];
        if (!any) return;
    }
    const int ncol = t.nu * t.nr;
    if (a.flops && threadIdx.x == 0) {
        int cols = 0;
        for (int c = 0; c < ncol; ++c) cols += (a.active == nullptr || a.active[t.r0 + c % t.nr]) ? 1 : 0;
        const int r_lo = max(lo, row0), r_hi = min(min(hi, row0 + BMT), a.M);
        atomicAdd(a.flops, 2ULL * (unsigned long long)max(0, r_hi - r_lo) * (unsigned long long)a.K *
                               (unsigned long long)cols);
    }
    const TM* __restrict__ A = reinterpret_cast<const TM*>(a.mats) + (long long)t.mat * a.mat_stride;
    const int tid = threadIdx.x;
    const int tr = tid / CG, tc = tid % CG;    // row 0..BMT-1, column group 0..CG-1
    TM acc[4] = {TM(0), TM(0), TM(0), TM(0)};
    double acc_lo[4] = {0.0, 0.0, 0.0, 0.0};   // EPI 3: running error of acc

    const double* colp[(BNT * BK) / GT];
#pragma unroll
    for (int l = 0; l < (BNT * BK) / GT; ++l) {
        const int e = tid + l * GT, c = e >> 4;
        colp[l] = nullptr;
        if (c < ncol) {
            const int u = t.u0 + c / t.nr, r = t.r0 + c % t.nr;
            colp[l] = a.in + (long long)r * a.in_rs + (long long)u * a.in_us + a.in_off + t.off;
        }
    }
    for (int k0 = 0; k0 < a.K; k0 += BK) {
        for (int e = tid; e < BMT * BK; e += GT) {
            const int i = e >> 4, kk = e & 15;
            const int row = row0 + i, k = k0 + kk;
            As[kk][i] = (row < a.M && k < a.K) ? A[(long long)row * a.K + k] : TM(0);
        }
#pragma unroll
        for (int l = 0; l < (BNT * BK) / GT; ++l) {
            const int e = tid + l * GT, c = e >> 4, kk = e & 15;
            const int k = k0 + kk;
            Bs[kk][c] = (colp[l] != nullptr && k < a.K) ? TM(colp[l][k]) : TM(0);
        }
        __syncthreads();
        if (EPI == 3) {
            // compensated dot products (Ogita, Rump & Oishi, "Accurate sum and
            // dot product", 2005, Dot2): TwoProduct by FMA, TwoSum of the
            // running sum, both errors gathered in acc_lo
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const double av = (double)As[kk][tr];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // __dmul_rn / __dadd_rn / __dsub_rn are never contracted
                    // into FMAs, which the error-free transforms rely on
                    const double bv = (double)Bs[kk][tc * 4 + j];
                    const double p = __dmul_rn(av, bv);
                    const double pe = fma(av, bv, -p);
                    const double x = (double)acc[j];
                    const double sum = __dadd_rn(x, p);
                    const double bb = __dsub_rn(sum, x);
                    const double se = __dadd_rn(__dsub_rn(x, __dsub_rn(sum, bb)), __dsub_rn(p, bb));
                    acc[j] = (TM)sum;
                    acc_lo[j] += pe + se;
                }
            }
        } else if (k0 + BK <= a.K) {
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const TM av = As[kk][tr];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fma(av, Bs[kk][tc * 4 + j], acc[j]);
            }
        } else {   // last, partial slab
            const int kn = a.K - k0;
            for (int kk = 0; kk < kn; ++kk) {
                const TM av = As[kk][tr];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] = fma(av, Bs[kk][tc * 4 + j], acc[j]);
            }
        }
        __syncthreads();
    }
    const int row = row0 + tr;
    if (row < lo || row >= hi || row >= a.M) return;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = tc * 4 + j;
        if (c >= ncol) continue;
        const int u = t.u0 + c / t.nr, r = t.r0 + c % t.nr;
        if (a.active && !a.active[r]) continue;
        const long long base = (long long)r * a.out_rs + (long long)u * a.out_us + t.off;
        const long long addr = base + (row < a.msplit ? a.out_off0 + row : a.out_off1 + (row - a.msplit));
        double v = (double)acc[j];
        if (EPI == 3) {   // (hi, lo) = add + acc + acc_lo, TwoSum for the first addition
            const double x = a.add[addr];
            const double sum = __dadd_rn(x, v);
            const double bb = __dsub_rn(sum, x);
            const double se = __dadd_rn(__dsub_rn(x, __dsub_rn(sum, bb)), __dsub_rn(v, bb));
            a.out[addr] = sum;
            a.out_lo[addr] = se + acc_lo[j];
            continue;
        }
        if (EPI == 1) v += a.add[addr];
        a.out[addr] = v;
    }
}

template <int EPI, typename TM, int BMT = BM>
__global__ void __launch_bounds__(GT) class_gemm_kernel(GemmArgs a, const Tile* __restrict__ tiles) {
    constexpr int BNT = 4 * GT / BMT;
    __shared__ TM As[BK][BMT + 1];
    __shared__ __align__(16) TM Bs[BK][BNT + 4];
    // 1-D grid, the row tiles of a column tile consecutive: the tile's input
    // columns are read by all its row tiles while they are still in L2
    const int nrow = (a.M + BMT - 1) / BMT, tile = blockIdx.x / nrow;
    class_gemm_tile<EPI, TM, BMT>(a, tiles[tile], blockIdx.x - tile * nrow, &As[0][0], &Bs[0][0]);
}

// ---------------------------------------------------------------------------
// Mirror form of the class GEMM.  With uniform h_x an interior strip, and an
// interior block-Jacobi pair, is symmetric under the reflection of x about its
// centre: with J the reversal of the order of the nb faces of a column (each
// face of fz values keeps its z order), the class matrix has J Mat J = Mat.
// Let h = nb fz / 2, v1 the first half of a column and v2' = (J v)[0:h] the
// reflected second half, X = Mat[0:h, 0:h] and N[i][j] = Mat[i][mirror(j)].
// Then (Mat v)[0:h] = X v1 + N v2' and (Mat v)[mirror(i)] = (N v1 + X v2')[i],
// so with s = v1 + v2', d = v1 - v2' and Hp, Hm = (X +- N) / 2:
//     out[i] = (Hp s + Hm d)[i],   out[mirror(i)] = (Hp s - Hm d)[i],
// two h x h products instead of one 2h x 2h product: half the FLOPs.  mats
// holds [Hp; Hm] per matrix, M = K = h, nb = 2 (Schur blocks G, one face per
// half) or 4 (block-Jacobi pairs).  The same split holds for any involution
// of the index set that commutes with Mat (first-half positions p(k), their
// images q(k)): nb = -1 or -2 is the z-reversal inside each block of f_z
// values, a symmetry of every slot inverse (L_z + s I)^-1 of the fast strip
// solver when h_z is uniform.  The output addressing (msplit, out_off0/1)
// and the epilogues (EPI 0 store, EPI 1 add) are those of class_gemm_kernel.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int mirror_index(int i, int fz, int rev) {
    return rev + i - (i >= fz ? 2 * fz : 0);   // (nb - 1 - i / fz) fz + i % fz for i < 2 fz
}

// The index pair (p, q) of half-index k: mirror_nb > 0 reverses the order of
// the faces (p = k, q = the mirrored face position); mirror_nb < 0 reverses the
// nodes inside each of -mirror_nb blocks of `face` values (the z-reversal of a
// slot matrix of the fast strip solver: p runs over the first half of every
// block, q is its reflection in the block).
__device__ __forceinline__ void mirror_pq(int k, int nb, int face, int rev, int& p, int& q) {
    if (nb > 0) {
        p = k;
        q = mirror_index(k, face, rev);
    } else {
        const int hb = face >> 1, b = k / hb, z = k - b * hb;
        p = b * face + z;
        q = b * face + face - 1 - z;
    }
}

// One output tile of the mirror form (two A slabs and two B slabs).
template <int EPI, typename TM, int BMT>
__device__ __forceinline__ void mirror_gemm_tile(const GemmArgs& a, const Tile t, int by, TM* A_, TM* B_) {
    constexpr int BNT = 4 * GT / BMT;
    constexpr int CG = GT / BMT;
    auto Ap = reinterpret_cast<TM (*)[BMT + 1]>(A_);
    auto Am = reinterpret_cast<TM (*)[BMT + 1]>(A_ + BK * (BMT + 1));
    auto Bp = reinterpret_cast<TM (*)[BNT + 4]>(__builtin_assume_aligned(B_, 16));
    auto Bm = reinterpret_cast<TM (*)[BNT + 4]>(__builtin_assume_aligned(B_ + BK * (BNT + 4), 16));
    const int row0 = by * BMT;
    const int h = a.M;
    if (row0 >= h) return;
    if (a.active) {
        int any = 0;
        for (int c = 0; c < t.nr; ++c) any |= a.active[t.r0 + c];
        if (!any) return;
    }
    const int ncol = t.nu * t.nr;
    if (a.flops && threadIdx.x == 0) {
        int cols = 0;
        for (int c = 0; c < ncol; ++c) cols += (a.active == nullptr || a.active[t.r0 + c % t.nr]) ? 1 : 0;
        const int rows = min(h, row0 + BMT) - row0;
        atomicAdd(a.flops, 4ULL * (unsigned long long)rows * (unsigned long long)h * (unsigned long long)cols);
    }
    const TM* __restrict__ Hp = reinterpret_cast<const TM*>(a.mats) + (long long)t.mat * a.mat_stride;
    const TM* __restrict__ Hm = Hp + (long long)h * h;
    const int nbm = a.mirror_nb, fz = a.face, rev = (a.mirror_nb - 1) * a.face;
    const int tid = threadIdx.x;
    const int tr = tid / CG, tc = tid % CG;
    TM accp[4] = {TM(0), TM(0), TM(0), TM(0)};
    TM accm[4] = {TM(0), TM(0), TM(0), TM(0)};
    const bool live = row0 + tr < h;

    const double* colp[(BNT * BK) / GT];
#pragma unroll
    for (int l = 0; l < (BNT * BK) / GT; ++l) {
        const int e = tid + l * GT, c = e >> 4;
        colp[l] = nullptr;
        if (c < ncol) {
            const int u = t.u0 + c / t.nr, r = t.r0 + c % t.nr;
            colp[l] = a.in + (long long)r * a.in_rs + (long long)u * a.in_us + a.in_off + t.off;
        }
    }
    for (int k0 = 0; k0 < h; k0 += BK) {
        for (int e = tid; e < BMT * BK; e += GT) {
            const int i = e >> 4, kk = e & 15;
            const int row = row0 + i, k = k0 + kk;
            const bool ok = row < h && k < h;
            Ap[kk][i] = ok ? Hp[(long long)row * h + k] : TM(0);
            Am[kk][i] = ok ? Hm[(long long)row * h + k] : TM(0);
        }
#pragma unroll
        for (int l = 0; l < (BNT * BK) / GT; ++l) {
            const int e = tid + l * GT, c = e >> 4, kk = e & 15;
            const int k = k0 + kk;
            TM sp = TM(0), sm = TM(0);
            if (colp[l] != nullptr && k < h) {
                int pk, qk;
                mirror_pq(k, nbm, fz, rev, pk, qk);
                const double v1 = colp[l][pk], v2 = colp[l][qk];
                sp = TM(v1 + v2);
                sm = TM(v1 - v2);
            }
            Bp[kk][c] = sp;
            Bm[kk][c] = sm;
        }
        __syncthreads();
        if (!live) {
            // padded row of the last row tile: its products are never stored
            // (warp-uniform where h is a multiple of the rows a warp covers)
        } else if (k0 + BK <= h) {
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                const TM ap = Ap[kk][tr], am = Am[kk][tr];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    accp[j] = fma(ap, Bp[kk][tc * 4 + j], accp[j]);
                    accm[j] = fma(am, Bm[kk][tc * 4 + j], accm[j]);
                }
            }
        } else {   // last, partial slab
            const int kn = h - k0;
            for (int kk = 0; kk < kn; ++kk) {
                const TM ap = Ap[kk][tr], am = Am[kk][tr];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    accp[j] = fma(ap, Bp[kk][tc * 4 + j], accp[j]);
                    accm[j] = fma(am, Bm[kk][tc * 4 + j], accm[j]);
                }
            }
        }
        __syncthreads();
    }
    int row = row0 + tr;
    if (row >= h) return;
    int mrow;
    mirror_pq(row, nbm, fz, rev, row, mrow);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = tc * 4 + j;
        if (c >= ncol) continue;
        const int u = t.u0 + c / t.nr, r = t.r0 + c % t.nr;
        if (a.active && !a.active[r]) continue;
        const long long base = (long long)r * a.out_rs + (long long)u * a.out_us + t.off;
        const long long a1 = base + (row < a.msplit ? a.out_off0 + row : a.out_off1 + (row - a.msplit));
        const long long a2 = base + (mrow < a.msplit ? a.out_off0 + mrow : a.out_off1 + (mrow - a.msplit));
        double y1 = (double)accp[j] + (double)accm[j];
        double y2 = (double)accp[j] - (double)accm[j];
        if (EPI == 1) {
            y1 += a.add[a1];
            y2 += a.add[a2];
        }
        a.out[a1] = y1;
        a.out[a2] = y2;
    }
}

template <int EPI, typename TM, int BMT>
__global__ void __launch_bounds__(GT) mirror_gemm_kernel(GemmArgs a, const Tile* __restrict__ tiles) {
    constexpr int BNT = 4 * GT / BMT;
    __shared__ TM Ap[2][BK][BMT + 1];
    __shared__ __align__(16) TM Bp[2][BK][BNT + 4];
    const int nrow = (a.M + BMT - 1) / BMT, tile = blockIdx.x / nrow;
    mirror_gemm_tile<EPI, TM, BMT>(a, tiles[tile], blockIdx.x - tile * nrow, &Ap[0][0][0], &Bp[0][0][0]);
}

template <int BMT>
static void launch_shape(const GemmArgs& a, const Tile* d_tiles, int ntiles, int epi, cudaStream_t s) {
    dim3 grid(ntiles * ((a.M + BMT - 1) / BMT));
    if (a.mirror_nb != 0) {
        if (a.fp32 && epi == 1)
            mirror_gemm_kernel<1, float, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
        else if (a.fp32)
            mirror_gemm_kernel<0, float, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
        else if (epi == 1)
            mirror_gemm_kernel<1, double, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
        else
            mirror_gemm_kernel<0, double, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
        return;
    }
    if (a.fp32 && epi == 1)
        class_gemm_kernel<1, float, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
    else if (a.fp32)
        class_gemm_kernel<0, float, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
    else if (epi == 1)
        class_gemm_kernel<1, double, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
    else if (epi == 3)
        class_gemm_kernel<3, double, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
    else
        class_gemm_kernel<0, double, BMT><<<grid, GT, 0, s>>>(a, d_tiles);
}

int gemm_tile_columns(int shape) { return shape == 1 ? 64 : 32; }

void launch_class_gemm(const GemmArgs& a, const Tile* d_tiles, int ntiles, int epi, void* stream) {
    if (ntiles <= 0) return;
    cudaStream_t s = (cudaStream_t)stream;
    if (a.shape == 1)
        launch_shape<8>(a, d_tiles, ntiles, epi, s);
    else
        launch_shape<16>(a, d_tiles, ntiles, epi, s);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Deflation (Sec. 3.3)
// ---------------------------------------------------------------------------

// gate: 0 -> rhs running Arnoldi (active), 1 -> rhs not yet converged
__device__ __forceinline__ bool gate_ok(const KArgs& a, int r, int gate) {
    return gate == 0 ? a.active[r] != 0 : a.done[r] == 0;
}

// Z^T (v - vsub) for right-hand side r: one warp per deflation group, NT
// threads per (virtual) block bx.
template <int NT>
__device__ __forceinline__ void deflate_sum_body(const KArgs& a, const double* __restrict__ v,
                                                 const double* __restrict__ vsub, int gate, int bx, int r) {
    if (!gate_ok(a, r, gate)) return;
    const int wg = (bx * NT + (int)threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wg >= a.d) return;
    const int t = wg / a.ng, gi = wg % a.ng, gs = a.fz / a.ng;
    const long long off = (long long)r * a.ld + (long long)(2 * t + 1) * a.fz + (long long)gi * gs;
    double s = 0.0;
    for (int z = lane; z < gs; z += 32) {
        double x = v[off + z] + v[off + a.fz + z];
        if (vsub) x -= vsub[off + z] + vsub[off + a.fz + z];
        s += x;
    }
    s = warp_sum(s);
    if (lane == 0) a.q[(long long)r * a.d + wg] = s;
}

__global__ void deflate_sum_kernel(KArgs a, const double* __restrict__ v, const double* __restrict__ vsub,
                                   int gate) {
    deflate_sum_body<VB>(a, v, vsub, gate, blockIdx.x, blockIdx.y);
}

static void deflate_sum_gate(const KArgs& a, const double* v, const double* vsub, int gate, cudaStream_t s) {
    dim3 grid((a.d * 32 + VB - 1) / VB, a.R);
    deflate_sum_kernel<<<grid, VB, 0, s>>>(a, v, vsub, gate);
    count_launches(1);
}

void k_deflate_sum(const KArgs& a, const double* v, const double* vsub, cudaStream_t s) {
    deflate_sum_gate(a, v, vsub, 0, s);
}

// c = K q for right-hand side r: one warp per coarse row.
template <int NT>
__device__ __forceinline__ void coarse_body(const KArgs& a, int gate, int bx, int r) {
    if (!gate_ok(a, r, gate)) return;
    const int i = (bx * NT + (int)threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (i >= a.d) return;
    if (!a.K) {                       // no deflation (the outer flexible GMRES of the nested form)
        if (lane == 0) a.c[(long long)r * a.d + i] = 0.0;
        return;
    }
    const double* K = a.K + (long long)a.op[r] * a.K_stride + (long long)i * a.d;
    const double* q = a.q + (long long)r * a.d;
    double s = 0.0;
    for (int j = lane; j < a.d; j += 32) s = fma(K[j], q[j], s);
    s = warp_sum(s);
    if (lane == 0) a.c[(long long)r * a.d + i] = s;
}

__global__ void coarse_kernel(KArgs a, int gate) {
    coarse_body<VB>(a, gate, blockIdx.x, blockIdx.y);
}

void k_coarse(const KArgs& a, cudaStream_t s) {
    dim3 grid((a.d * 32 + VB - 1) / VB, a.R);
    coarse_kernel<<<grid, VB, 0, s>>>(a, 0);
    count_launches(1);
}
static void k_coarse_gate(const KArgs& a, int gate, cudaStream_t s) {
    dim3 grid((a.d * 32 + VB - 1) / VB, a.R);
    coarse_kernel<<<grid, VB, 0, s>>>(a, gate);
    count_launches(1);
}

// (S Z c) at face-vector position e (Sec. 3.3): Z c is c_{t,g} on both faces of
// interface t; S adds the G row-sums rho of the two strips that touch it.
__device__ __forceinline__ double szc_at(const KArgs& a, int r, long long e) {
    const int fz = a.fz;
    const int F = (int)(e / fz), Z = (int)(e - (long long)F * fz);
    if (F == 0 || F >= 2 * a.mx - 1) return 0.0;
    const int i = F >> 1, s = F & 1, ng = a.ng, gs = fz / ng;
    const double* c = a.c + (long long)r * a.d;
    const double* rho = a.rho + (long long)a.op[r] * a.rho_stride;
    const long long fz2 = 2LL * fz;
    double val;
    if (s == 1) {  // east face of strip i, interface t = i; strip i+1's west output half
        const int t = i, cl = a.strip_cls[i + 1];
        val = c[t * ng + Z / gs];
        const double* rL = rho + (long long)(cl * 2 + 0) * ng * fz2;
        const double* rR = rho + (long long)(cl * 2 + 1) * ng * fz2;
        const bool has_next = (t + 1) <= a.mx - 2;
        for (int gg = 0; gg < ng; ++gg) {
            val = fma(c[t * ng + gg], rL[gg * fz2 + Z], val);
            if (has_next) val = fma(c[(t + 1) * ng + gg], rR[gg * fz2 + Z], val);
        }
    } else {       // west face of strip i, interface t = i-1; strip i-1's east output half
        const int t = i - 1, cl = a.strip_cls[i - 1];
        val = c[t * ng + Z / gs];
        const double* rL = rho + (long long)(cl * 2 + 0) * ng * fz2 + fz;
        const double* rR = rho + (long long)(cl * 2 + 1) * ng * fz2 + fz;
        const bool has_prev = t >= 1;
        for (int gg = 0; gg < ng; ++gg) {
            if (has_prev) val = fma(c[(t - 1) * ng + gg], rL[gg * fz2 + Z], val);
            val = fma(c[t * ng + gg], rR[gg * fz2 + Z], val);
        }
    }
    return val;
}

// Z c at position e (prolongation of the coarse vector).
__device__ __forceinline__ double zc_at(const KArgs& a, int r, long long e) {
    const int fz = a.fz;
    const int F = (int)(e / fz), Z = (int)(e - (long long)F * fz);
    if (F == 0 || F >= 2 * a.mx - 1) return 0.0;
    const int t = (F - 1) >> 1, gs = fz / a.ng;
    return a.c[(long long)r * a.d + t * a.ng + Z / gs];
}

// ---------------------------------------------------------------------------
// CGS2 Arnoldi step (Sec. 3.1 orthogonalisation; CGS applied twice)
// ---------------------------------------------------------------------------
// Chunk bx of right-hand side r; sm: ch + m + 2 + 32 doubles of shared memory.
// T: the arithmetic of the projections and dot products (storage stays FP64);
// float for the inner solve of the nested mixed-precision form (a.f32).
template <int NT, typename T = double>
__device__ __forceinline__ void cgs_body(const KArgs& a, int j, int mode, int bx, int r, double* sm) {
    if (!a.active[r]) return;
    double* wsh = sm;                 // [ch]
    double* hsh = sm + a.ch;          // [m+2]
    double* red = hsh + (a.m + 2);    // [32]
    const long long e0 = (long long)bx * a.ch;
    const long long e1 = min(e0 + (long long)a.ch, a.kp);
    const int len = (int)(e1 - e0);
    double* w = a.w + (long long)r * a.ld;
    const double* Vr = a.V + (long long)r * (a.m + 1) * a.ld;
    const int nv = j + 1;
    const long long pstride = (long long)a.nch * (a.m + 2);
    if (mode == 0) {
        for (int e = threadIdx.x; e < len; e += NT) {
            double x = w[e0 + e] - szc_at(a, r, e0 + e);
            wsh[e] = x;
            w[e0 + e] = x;
        }
    } else {
        const double* pin = (mode == 1 ? a.part1 : a.part2) + (long long)r * pstride;
        for (int i = threadIdx.x; i < nv; i += NT) {
            double s = 0.0;
            for (int ch = 0; ch < a.nch; ++ch) s += pin[(long long)ch * (a.m + 2) + i];
            hsh[i] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < len; e += NT) {
            T x = (T)w[e0 + e];
            for (int i = 0; i < nv; ++i) x = fma(-(T)Vr[(long long)i * a.ld + e0 + e], (T)hsh[i], x);
            wsh[e] = (double)x;
            w[e0 + e] = (double)x;
        }
        if (bx == 0) {
            if (mode == 1)
                for (int i = threadIdx.x; i < nv; i += NT) a.htmp[(long long)r * (a.m + 1) + i] = hsh[i];
            else
                for (int i = threadIdx.x; i < nv; i += NT)
                    a.Hc[((long long)r * a.m + j) * (a.m + 1) + i] = a.htmp[(long long)r * (a.m + 1) + i] + hsh[i];
        }
    }
    __syncthreads();
    if (mode <= 1) {
        double* pout = (mode == 0 ? a.part1 : a.part2) + (long long)r * pstride + (long long)bx * (a.m + 2);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int i = wid; i < nv; i += NT / 32) {
            const double* vi = Vr + (long long)i * a.ld + e0;
            T s = T(0);
            for (int e = lane; e < len; e += 32) s = fma((T)vi[e], (T)wsh[e], s);
            s = warp_sum(s);
            if (lane == 0) pout[i] = (double)s;
        }
    } else {
        T st = T(0);
        for (int e = threadIdx.x; e < len; e += NT) st = fma((T)wsh[e], (T)wsh[e], st);
        double s = block_sum<NT>((double)st, red);
        if (threadIdx.x == 0) a.part1[(long long)r * pstride + (long long)bx * (a.m + 2)] = s;
    }
}

__global__ void __launch_bounds__(VB) cgs_kernel(KArgs a, int j, int mode) {
    extern __shared__ double sm[];
    if (a.f32)
        cgs_body<VB, float>(a, j, mode, blockIdx.x, blockIdx.y, sm);
    else
        cgs_body<VB, double>(a, j, mode, blockIdx.x, blockIdx.y, sm);
}

// Concatenated Krylov spaces (a.grp > 1): the partial sums of chunk blockIdx.x,
// slots [0, nslots), summed over the columns of group blockIdx.y that take part
// (gate 0: active, gate 1: not done) and written back to each of them, so that
// every column's reduction over chunks yields the dot product (or norm) of the
// concatenated vectors.  Columns are summed in index order (deterministic).
__global__ void group_partials_kernel(KArgs a, double* __restrict__ part, int nslots, int gate) {
    const int ch = blockIdx.x;
    const int r0 = blockIdx.y * a.grp, r1 = min(r0 + a.grp, a.R);
    const long long pstride = (long long)a.nch * (a.m + 2);
    const long long off = (long long)ch * (a.m + 2);
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) {
        double sum = 0.0;
        for (int r = r0; r < r1; ++r)
            if (gate == 0 ? a.active[r] != 0 : a.done[r] == 0) sum += part[(long long)r * pstride + off + i];
        for (int r = r0; r < r1; ++r)
            if (gate == 0 ? a.active[r] != 0 : a.done[r] == 0) part[(long long)r * pstride + off + i] = sum;
    }
}

static void group_partials(const KArgs& a, double* part, int nslots, int gate, cudaStream_t s) {
    if (a.grp <= 1) return;
    dim3 grid(a.nch, (a.R + a.grp - 1) / a.grp);
    group_partials_kernel<<<grid, 64, 0, s>>>(a, part, nslots, gate);
    count_launches(1);
}

void k_cgs(const KArgs& a, int j, int mode, cudaStream_t s) {
    dim3 grid(a.nch, a.R);
    size_t sh = (size_t)(a.ch + a.m + 2 + 32) * sizeof(double);
    cgs_kernel<<<grid, VB, sh, s>>>(a, j, mode);
    count_launches(1);
    // mode 0 leaves the first pass's dots in part1, mode 1 the second pass's in
    // part2, mode 2 the squared norm in part1 slot 0
    group_partials(a, mode == 1 ? a.part2 : a.part1, mode == 2 ? 1 : j + 1, 0, s);
}

template <int NT = VB>
__device__ double reduce_part(const KArgs& a, int r, int slot, double* red) {
    const long long pstride = (long long)a.nch * (a.m + 2);
    const double* p = a.part1 + (long long)r * pstride;
    double s = 0.0;
    for (int ch = threadIdx.x; ch < a.nch; ch += NT) s += p[(long long)ch * (a.m + 2) + slot];
    return block_sum<NT>(s, red);
}

// beta = ||w||, V[j+1] = w / beta over chunk bx, and (block bx = 0) the Givens
// update of the Hessenberg column and the convergence flags of rhs r.
template <int NT>
__device__ __forceinline__ void normalize_body(const KArgs& a, int j, int last_allowed, int bx, int r, double* red) {
    if (!a.active[r]) return;
    const double beta = sqrt(reduce_part<NT>(a, r, 0, red));
    const bool bad = !(beta > 1e-300) || !isfinite(beta);
    const long long e0 = (long long)bx * a.ch;
    const long long e1 = min(e0 + (long long)a.ch, a.kp);
    const double* w = a.w + (long long)r * a.ld;
    double* vn = a.V + ((long long)r * (a.m + 1) + (j + 1)) * a.ld;
    const double inv = bad ? 0.0 : 1.0 / beta;
    for (long long e = e0 + threadIdx.x; e < e1; e += NT) vn[e] = w[e] * inv;
    if (bx == 0 && threadIdx.x == 0) {
        double* h = a.Hc + ((long long)r * a.m + j) * (a.m + 1);
        double* cs = a.cs + (long long)r * a.m;
        double* sn = a.sn + (long long)r * a.m;
        double* g = a.gv + (long long)r * (a.m + 1);
        h[j + 1] = isfinite(beta) ? beta : 0.0;
        for (int i = 0; i < j; ++i) {
            const double t = cs[i] * h[i] + sn[i] * h[i + 1];
            h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
            h[i] = t;
        }
        const double rho = hypot(h[j], h[j + 1]);
        double c = 1.0, s = 0.0;
        if (rho > 0.0) { c = h[j] / rho; s = h[j + 1] / rho; }
        h[j] = rho;
        h[j + 1] = 0.0;
        cs[j] = c;
        sn[j] = s;
        g[j + 1] = -s * g[j];
        g[j] = c * g[j];
        a.nit[r] = j + 1;
        if (a.hist) {
            const int k = a.hist_base[r] + j + 1;
            if (k < a.hist_stride) a.hist[(long long)r * a.hist_stride + k] = fabs(g[j + 1]) / a.bnorm[r];
        }
        const bool nonfinite = !isfinite(g[j + 1]) || !isfinite(rho);
        if (nonfinite || !(rho > 0.0)) a.flags[r] |= 1;
        if (nonfinite || !(rho > 0.0) || fabs(g[j + 1]) <= a.target[r] || j + 1 >= last_allowed || bad)
            a.active[r] = 0;
    }
}

__global__ void __launch_bounds__(VB) normalize_kernel(KArgs a, int j, int last_allowed) {
    __shared__ double red[32];
    normalize_body<VB>(a, j, last_allowed, blockIdx.x, blockIdx.y, red);
}

void k_normalize(const KArgs& a, int j, int last_allowed, cudaStream_t s) {
    dim3 grid(a.nch, a.R);
    normalize_kernel<<<grid, VB, 0, s>>>(a, j, last_allowed);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Persistent Arnoldi kernel: every step of a restart cycle (block-Jacobi
// apply, Schur product, deflation restriction and coarse product, the three
// CGS2 passes, normalisation and Givens update) for every active right-hand
// side in one cooperative launch.  Each phase is the work of one of the
// launches above, spread over the resident blocks as virtual blocks; phases
// are separated by a grid-wide barrier whose every wait has a time limit:
// a block that waits longer sets *status and all blocks leave at their next
// barrier (no block ever spins without bound).
// ---------------------------------------------------------------------------
static constexpr int PT = GT;   // threads of a persistent block (one GEMM tile each)

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier number `epoch` (counted from 1): arrive on the counter,
// wait until every block of the grid (one more under the stall test) has
// arrived.  Returns false when this block, or another one, gave up.
__device__ bool grid_barrier(const PersistArgs& p, unsigned int epoch, int* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int target = epoch * gridDim.x + (p.stall ? 1u : 0u);
        int ok = 1;
        __threadfence();
        atomicAdd(p.bar, 1u);
        const unsigned long long t0 = global_ns();
        unsigned int spins = 0;
        while (ld_acquire_u32(p.bar) < target) {
            if (*(volatile int*)p.status != 0) { ok = 0; break; }
            if ((++spins & 31u) == 0 && global_ns() - t0 > (unsigned long long)p.wait_ns) {
                atomicCAS(p.status, 0, 1);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

// One tile of a dense product, dispatched on precision, form, epilogue and
// tile shape; sm: the block's shared memory (16-byte aligned).
__device__ __forceinline__ void pgemm_tile(const GemmArgs& a, const Tile t, int by, int epi, double* sm) {
    if (a.mirror_nb != 0) {
        if (a.fp32) {
            float* f = reinterpret_cast<float*>(sm);
            if (a.shape == 1) {
                if (epi) mirror_gemm_tile<1, float, 8>(a, t, by, f, f + 2 * BK * 9);
                else mirror_gemm_tile<0, float, 8>(a, t, by, f, f + 2 * BK * 9);
            } else {
                if (epi) mirror_gemm_tile<1, float, 16>(a, t, by, f, f + 2 * BK * 17);
                else mirror_gemm_tile<0, float, 16>(a, t, by, f, f + 2 * BK * 17);
            }
        } else {
            if (a.shape == 1) {
                if (epi) mirror_gemm_tile<1, double, 8>(a, t, by, sm, sm + 2 * BK * 9);
                else mirror_gemm_tile<0, double, 8>(a, t, by, sm, sm + 2 * BK * 9);
            } else {
                if (epi) mirror_gemm_tile<1, double, 16>(a, t, by, sm, sm + 2 * BK * 17);
                else mirror_gemm_tile<0, double, 16>(a, t, by, sm, sm + 2 * BK * 17);
            }
        }
        return;
    }
    if (a.fp32) {
        float* f = reinterpret_cast<float*>(sm);
        if (a.shape == 1) {
            if (epi) class_gemm_tile<1, float, 8>(a, t, by, f, f + BK * 9);
            else class_gemm_tile<0, float, 8>(a, t, by, f, f + BK * 9);
        } else {
            if (epi) class_gemm_tile<1, float, 16>(a, t, by, f, f + BK * 17);
            else class_gemm_tile<0, float, 16>(a, t, by, f, f + BK * 17);
        }
    } else {
        if (a.shape == 1) {
            if (epi) class_gemm_tile<1, double, 8>(a, t, by, sm, sm + BK * 9);
            else class_gemm_tile<0, double, 8>(a, t, by, sm, sm + BK * 9);
        } else {
            if (epi) class_gemm_tile<1, double, 16>(a, t, by, sm, sm + BK * 17);
            else class_gemm_tile<0, double, 16>(a, t, by, sm, sm + BK * 17);
        }
    }
}

// The tiles of n product launches as one list of virtual blocks; the row
// tiles of a column tile are consecutive (its input columns are read while
// they are still in L2).  in_add shifts every launch's input offset.
__device__ void gemm_phase(const PGemm* g, int n, long long in_add, double* sm) {
    int total = 0;
    for (int i = 0; i < n; ++i) total += g[i].ntiles * g[i].nrow;
    for (int v = blockIdx.x; v < total; v += gridDim.x) {
        int i = 0, vv = v;
        while (vv >= g[i].ntiles * g[i].nrow) {
            vv -= g[i].ntiles * g[i].nrow;
            ++i;
        }
        GemmArgs a = g[i].a;
        a.in_off += in_add;
        const int tile = vv / g[i].nrow, by = vv - tile * g[i].nrow;
        pgemm_tile(a, g[i].tiles[tile], by, g[i].epi, sm);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(PT, 4) arnoldi_persistent_kernel(PersistArgs p) {
    extern __shared__ __align__(16) double psm[];
    __shared__ int flag;
    const KArgs& a = p.ka;
    unsigned int epoch = 0;
    const int ngx = (a.d * 32 + PT - 1) / PT;       // virtual blocks per rhs of the deflation phases
    for (int j = p.j0; j < p.last_allowed; ++j) {
        const int set = (p.use_fp32 && j >= p.fp64_steps) ? 1 : 0;
        gemm_phase(p.bj[set], p.nbj[set], (long long)j * p.bj_step, psm);          // z = M^-1 v_j
        if (!grid_barrier(p, ++epoch, &flag)) return;
        gemm_phase(p.sc, p.nsc, 0, psm);                                           // w = S z
        if (p.Zb) {                                                                // FGMRES keeps z_j
            const long long n = (long long)a.R * a.kp;
            for (long long e = (long long)blockIdx.x * PT + threadIdx.x; e < n; e += (long long)gridDim.x * PT) {
                const int r = (int)(e / a.kp);
                const long long i = e - (long long)r * a.kp;
                if (a.active[r]) p.Zb[(long long)r * a.m * a.ld + (long long)j * a.ld + i] = p.z[(long long)r * a.ld + i];
            }
        }
        if (!grid_barrier(p, ++epoch, &flag)) return;
        for (int v = blockIdx.x; v < ngx * a.R; v += gridDim.x) deflate_sum_body<PT>(a, a.w, nullptr, 0, v % ngx, v / ngx);
        if (!grid_barrier(p, ++epoch, &flag)) return;
        for (int v = blockIdx.x; v < ngx * a.R; v += gridDim.x) coarse_body<PT>(a, 0, v % ngx, v / ngx);
        if (!grid_barrier(p, ++epoch, &flag)) return;
        for (int mode = 0; mode < 3; ++mode) {
            for (int v = blockIdx.x; v < a.nch * a.R; v += gridDim.x) {
                cgs_body<PT>(a, j, mode, v % a.nch, v / a.nch, psm);
                __syncthreads();
            }
            if (!grid_barrier(p, ++epoch, &flag)) return;
        }
        for (int v = blockIdx.x; v < a.nch * a.R; v += gridDim.x) {
            normalize_body<PT>(a, j, p.last_allowed, v % a.nch, v / a.nch, psm);
            __syncthreads();
        }
        if (!grid_barrier(p, ++epoch, &flag)) return;
        int any = 0;
        for (int r = 0; r < a.R; ++r) any |= *(volatile const int*)(a.active + r);
        if (!any) return;
    }
}

bool k_arnoldi_persistent(const PersistArgs& p, cudaStream_t s) {
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!coop) return false;
    // shared memory: the largest GEMM tile (mirror form, FP64, 8-row tiles)
    // or the CGS2 chunk buffer
    const size_t gemm_sm = sizeof(double) * 2 * (size_t)(BK * 9 + BK * (4 * GT / 8 + 4));
    const size_t cgs_sm = sizeof(double) * (size_t)(p.ka.ch + p.ka.m + 2 + 32);
    const size_t smem = gemm_sm > cgs_sm ? gemm_sm : cgs_sm;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, arnoldi_persistent_kernel, PT, smem) != cudaSuccess ||
        per_sm < 1)
        return false;
    // as many blocks as the largest phase has virtual blocks, at most what
    // fits on the device (a small problem keeps its barriers cheap)
    long long work = (long long)p.ka.nch * p.ka.R;
    work = std::max(work, (long long)((p.ka.d * 32 + PT - 1) / PT) * p.ka.R);
    for (int set = 0; set < 2; ++set) {
        long long t = 0;
        for (int i = 0; i < p.nbj[set]; ++i) t += (long long)p.bj[set][i].ntiles * p.bj[set][i].nrow;
        work = std::max(work, t);
    }
    long long tsc = 0;
    for (int i = 0; i < p.nsc; ++i) tsc += (long long)p.sc[i].ntiles * p.sc[i].nrow;
    work = std::max(work, tsc);
    const long long cap = (long long)per_sm * sms;
    PersistArgs q = p;
    void* args[] = {&q};
    const dim3 grid((unsigned)std::max(1LL, std::min(cap, work))), block(PT);
    if (cudaLaunchCooperativeKernel((const void*)arnoldi_persistent_kernel, grid, block, args, smem, s) != cudaSuccess)
        return false;
    count_launches(1);
    return true;
}

// Residual at the start of a restart cycle: r = (bS - s) - S Z c, c = K Z^T (bS - s).
__global__ void __launch_bounds__(VB) residual_kernel(KArgs a, const double* __restrict__ bS,
                                                     const double* __restrict__ sv) {
    const int r = blockIdx.y;
    if (a.done[r]) return;
    __shared__ double red[32];
    const long long e0 = (long long)blockIdx.x * a.ch;
    const long long e1 = min(e0 + (long long)a.ch, a.kp);
    const double* b = bS + (long long)r * a.ld;
    const double* sr = sv ? sv + (long long)r * a.ld : nullptr;
    double* v0 = a.V + (long long)r * (a.m + 1) * a.ld;
    double s2 = 0.0, b2 = 0.0, d2 = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += VB) {
        const double bb = b[e];
        double dd = bb - (sr ? sr[e] : 0.0);            // true residual b_S - S x_S
        if (sr && a.s_lo) dd = dd - a.s_lo[(long long)r * a.ld + e] - a.s_xlo[(long long)r * a.ld + e];
        const double x = dd - szc_at(a, r, e);          // deflated residual P d
        v0[e] = x;
        s2 = fma(x, x, s2);
        b2 = fma(bb, bb, b2);
        d2 = fma(dd, dd, d2);
    }
    s2 = block_sum(s2, red);
    b2 = block_sum(b2, red);
    d2 = block_sum(d2, red);
    if (threadIdx.x == 0) {
        const long long pstride = (long long)a.nch * (a.m + 2);
        double* p = a.part1 + (long long)r * pstride + (long long)blockIdx.x * (a.m + 2);
        p[0] = s2;
        p[1] = b2;
        p[2] = d2;
    }
}

void k_residual(const KArgs& a, const double* bS, const double* sv, cudaStream_t s) {
    deflate_sum_gate(a, bS, sv, 1, s);  // q = Z^T (bS - s) for every unconverged rhs
    k_coarse_gate(a, 1, s);
    dim3 grid(a.nch, a.R);
    residual_kernel<<<grid, VB, 0, s>>>(a, bS, sv);
    count_launches(1);
    group_partials(a, a.part1, 3, 1, s);   // ||P d||^2, ||b_S||^2, ||b_S - S x_S||^2
}

__global__ void __launch_bounds__(VB) cycle_start_kernel(KArgs a, double* __restrict__ c0, int stamp, double tol) {
    const int r = blockIdx.y;
    if (a.done[r]) return;
    __shared__ double red[32];
    const double beta = sqrt(reduce_part(a, r, 0, red));   // ||P d||: GMRES starting residual
    const double bn = sqrt(reduce_part(a, r, 1, red));     // ||b_S||
    const double dn = sqrt(reduce_part(a, r, 2, red));     // ||b_S - S x_S||: true residual
    const double target = (stamp == 1) ? tol * bn : a.target[r];
    const bool conv = (dn <= target) || !(bn > 0.0);
    const bool bad = !isfinite(beta) || !isfinite(dn);
    const bool lucky = !(beta > 0.0);                      // P d = 0: nothing left for GMRES
    const long long e0 = (long long)blockIdx.x * a.ch;
    const long long e1 = min(e0 + (long long)a.ch, a.kp);
    if (!(conv || bad || lucky)) {
        double* v0 = a.V + (long long)r * (a.m + 1) * a.ld;
        const double inv = 1.0 / beta;
        for (long long e = e0 + threadIdx.x; e < e1; e += VB) v0[e] *= inv;
    }
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < a.d; i += VB) c0[(long long)r * a.d + i] = a.c[(long long)r * a.d + i];
        if (threadIdx.x == 0) {
            if (stamp == 1) { a.target[r] = target; a.bnorm[r] = bn; }
            a.rnorm[r] = dn;
            a.nit[r] = 0;
            if (bad) a.flags[r] |= 1;
            if (conv || bad) {
                a.active[r] = 0;
            } else {
                double* g = a.gv + (long long)r * (a.m + 1);
                g[0] = beta;
                for (int i = 1; i <= a.m; ++i) g[i] = 0.0;
                a.active[r] = lucky ? 0 : 1;
            }
        }
    }
}

__global__ void commit_kernel(KArgs a, int stamp) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.R || a.done[r]) return;
    if (!a.active[r] && a.nit[r] == 0) a.done[r] = stamp;  // converged (or failed) at this cycle start
}

void k_cycle_start(const KArgs& a, double* c0, int first, double tol, cudaStream_t s) {
    dim3 grid(a.nch, a.R);
    // stamp == 1 marks the first cycle (targets are set from ||b_S||)
    cycle_start_kernel<<<grid, VB, 0, s>>>(a, c0, first ? 1 : 2, tol);
    count_launches(1);
    commit_kernel<<<(a.R + 127) / 128, 128, 0, s>>>(a, 1);
    count_launches(1);
}

// End of a cycle: x_S += t + Z (c0 - c), with t = M^-1 V y, c0 = K Z^T d from the
// cycle start and c = K Z^T S t (Q M^-1 y + Z C\ d restricted to this cycle).
__global__ void __launch_bounds__(VB) xs_update_kernel(KArgs a, double* __restrict__ xS, const double* __restrict__ t,
                                                      const double* __restrict__ c0) {
    const int r = blockIdx.y;
    if (a.done[r] || a.nit[r] <= 0) return;
    const long long e0 = (long long)blockIdx.x * a.ch;
    const long long e1 = min(e0 + (long long)a.ch, a.kp);
    const int fz = a.fz, gs = fz / a.ng;
    double* x = xS + (long long)r * a.ld;
    const double* tr = t + (long long)r * a.ld;
    for (long long e = e0 + threadIdx.x; e < e1; e += VB) {
        const int F = (int)(e / fz), Z = (int)(e - (long long)F * fz);
        double v = tr[e];
        if (F > 0 && F < 2 * a.mx - 1) {
            const long long ci = (long long)r * a.d + ((F - 1) >> 1) * a.ng + Z / gs;
            v += c0[ci] - a.c[ci];
        }
        if (a.xlo) {   // x_S = x + xlo: TwoSum, then renormalise (Fast2Sum)
            double* xl = a.xlo + (long long)r * a.ld;
            const double xv = x[e];
            const double sum = __dadd_rn(xv, v);
            const double bb = __dsub_rn(sum, xv);
            const double lo = __dadd_rn(xl[e], __dadd_rn(__dsub_rn(xv, __dsub_rn(sum, bb)), __dsub_rn(v, bb)));
            const double hi = __dadd_rn(sum, lo);
            xl[e] = __dsub_rn(lo, __dsub_rn(hi, sum));
            x[e] = hi;
        } else {
            x[e] += v;
        }
    }
}

void k_xs_update(const KArgs& a, double* xS, const double* t, const double* c0, cudaStream_t s) {
    dim3 grid(a.nch, a.R);
    xs_update_kernel<<<grid, VB, 0, s>>>(a, xS, t, c0);
    count_launches(1);
}

void k_deflate_coarse_pending(const KArgs& a, const double* v, cudaStream_t s) {
    deflate_sum_gate(a, v, nullptr, 1, s);
    k_coarse_gate(a, 1, s);
}

__global__ void __launch_bounds__(VB) cycle_update_kernel(KArgs a, double* __restrict__ Xp,
                                                         const double* __restrict__ basis, long long basis_rs) {
    const int r = blockIdx.y;
    if (a.done[r]) return;
    const int ni = a.nit[r];
    if (ni <= 0) return;
    extern __shared__ double y[];
    if (threadIdx.x == 0) {
        const double* g = a.gv + (long long)r * (a.m + 1);
        for (int i = ni - 1; i >= 0; --i) {
            double s = g[i];
            for (int l = i + 1; l < ni; ++l) s -= a.Hc[((long long)r * a.m + l) * (a.m + 1) + i] * y[l];
            const double d = a.Hc[((long long)r * a.m + i) * (a.m + 1) + i];
            y[i] = d != 0.0 ? s / d : 0.0;
        }
    }
    __syncthreads();
    const long long e0 = (long long)blockIdx.x * a.ch;
    const long long e1 = min(e0 + (long long)a.ch, a.kp);
    const double* Vr = basis + (long long)r * basis_rs;
    double* x = Xp + (long long)r * a.ld;
    for (long long e = e0 + threadIdx.x; e < e1; e += VB) {
        double s = 0.0;
        for (int i = 0; i < ni; ++i) s = fma(y[i], Vr[(long long)i * a.ld + e], s);
        x[e] = s;
    }
}

void k_cycle_update(const KArgs& a, double* Xp, cudaStream_t s, const double* basis, long long basis_rs) {
    dim3 grid(a.nch, a.R);
    if (!basis) {
        basis = a.V;
        basis_rs = (long long)(a.m + 1) * a.ld;
    }
    cycle_update_kernel<<<grid, VB, (size_t)(a.m + 1) * sizeof(double), s>>>(a, Xp, basis, basis_rs);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Full-grid kernels: RHS assembly, projections, recovery input, gauge
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(VB) rhs_assemble_kernel(GridArgs g, const double* __restrict__ f, long long f_ld,
                                                         const double* __restrict__ gb, long long g_ld,
                                                         double* __restrict__ b, long long b_ld,
                                                         const double* const* __restrict__ uL,
                                                         double* __restrict__ part, int nch, int ch) {
    const int r = blockIdx.y;
    __shared__ double red[32];
    const long long e0 = (long long)blockIdx.x * ch;
    const long long e1 = min(e0 + (long long)ch, g.r);
    const double* u = uL ? uL[r] : nullptr;
    const double* gr = gb ? gb + (long long)r * g_ld : nullptr;
    double s = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += VB) {
        double v = f[(long long)r * f_ld + e];
        if (gr) {
            const int X = (int)(e / g.fz), Z = (int)(e - (long long)X * g.fz);
            if (X == 0) v += g.tau_x * gr[Z];
            if (X == g.nx - 1) v += g.tau_x * gr[g.fz + Z];
            if (Z == 0) v += g.tau_z[0] * gr[2 * g.fz + X];
            if (Z == g.fz - 1) v += g.tau_z[g.mz - 1] * gr[2 * g.fz + g.nx + X];
        }
        b[(long long)r * b_ld + e] = v;
        if (u) s = fma(u[e], v, s);
    }
    if (u) {
        s = block_sum(s, red);
        if (threadIdx.x == 0) part[(long long)r * nch + blockIdx.x] = s;
    }
}

void k_rhs_assemble(const GridArgs& g, int R, const double* f, long long f_ld, const double* gb,
                    long long g_ld, double* b, long long b_ld, const double* const* uL,
                    double* part, int nch, int ch, cudaStream_t s) {
    dim3 grid(nch, R);
    rhs_assemble_kernel<<<grid, VB, 0, s>>>(g, f, f_ld, gb, g_ld, b, b_ld, uL, part, nch, ch);
    count_launches(1);
}

__global__ void __launch_bounds__(VB) dot_partial_kernel(long long len, const double* __restrict__ v, long long v_ld,
                                                        const double* const* __restrict__ u,
                                                        double* __restrict__ part, int nch, int ch) {
    const int r = blockIdx.y;
    const double* ur = u[r];
    if (!ur) return;
    __shared__ double red[32];
    const long long e0 = (long long)blockIdx.x * ch;
    const long long e1 = min(e0 + (long long)ch, len);
    double s = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += VB) s = fma(ur[e], v[(long long)r * v_ld + e], s);
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(long long)r * nch + blockIdx.x] = s;
}

void k_dot_partial(int R, long long len, const double* v, long long v_ld, const double* const* u,
                   double* part, int nch, int ch, cudaStream_t s) {
    dim3 grid(nch, R);
    dot_partial_kernel<<<grid, VB, 0, s>>>(len, v, v_ld, u, part, nch, ch);
    count_launches(1);
}

__global__ void __launch_bounds__(VB) project_kernel(long long len, double* __restrict__ v, long long v_ld,
                                                    const double* const* __restrict__ u,
                                                    const double* __restrict__ part, int nch, int ch) {
    const int r = blockIdx.y;
    const double* ur = u[r];
    if (!ur) return;
    __shared__ double red[32];
    double s = 0.0;
    for (int c = threadIdx.x; c < nch; c += VB) s += part[(long long)r * nch + c];
    s = block_sum(s, red);
    const long long e0 = (long long)blockIdx.x * ch;
    const long long e1 = min(e0 + (long long)ch, len);
    for (long long e = e0 + threadIdx.x; e < e1; e += VB) v[(long long)r * v_ld + e] -= s * ur[e];
}

void k_project(int R, long long len, double* v, long long v_ld, const double* const* u,
               const double* part, int nch, int ch, cudaStream_t s) {
    dim3 grid(nch, R);
    project_kernel<<<grid, VB, 0, s>>>(len, v, v_ld, u, part, nch, ch);
    count_launches(1);
}

__global__ void __launch_bounds__(VB) recovery_rhs_kernel(GridArgs g, const double* __restrict__ b, long long b_ld,
                                                         const double* __restrict__ xS, long long x_ld,
                                                         double* __restrict__ t2) {
    const int r = blockIdx.y;
    const long long e = (long long)blockIdx.x * VB + threadIdx.x;
    if (e >= g.r) return;
    const int X = (int)(e / g.fz), Z = (int)(e - (long long)X * g.fz);
    const int i = X / g.n, a = X - i * g.n;
    double v = b[(long long)r * b_ld + e];
    if (a == 0) v -= xS[(long long)r * x_ld + (long long)(2 * i) * g.fz + Z];
    if (a == g.N) v -= xS[(long long)r * x_ld + (long long)(2 * i + 1) * g.fz + Z];
    t2[(long long)r * g.r + e] = v;
}

void k_recovery_rhs(const GridArgs& g, int R, const double* b, long long b_ld, const double* xS,
                    long long x_ld, double* t2, cudaStream_t s) {
    dim3 grid((unsigned)((g.r + VB - 1) / VB), R);
    recovery_rhs_kernel<<<grid, VB, 0, s>>>(g, b, b_ld, xS, x_ld, t2);
    count_launches(1);
}

__global__ void __launch_bounds__(VB) gauge_partial_kernel(GridArgs g, const double* __restrict__ u, long long u_ld,
                                                          const int* __restrict__ apply,
                                                          double* __restrict__ part, int nch, int ch) {
    const int r = blockIdx.y;
    if (!apply[r]) return;
    __shared__ double red[32];
    const long long e0 = (long long)blockIdx.x * ch;
    const long long e1 = min(e0 + (long long)ch, g.r);
    double s = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += VB) {
        const int X = (int)(e / g.fz), Z = (int)(e - (long long)X * g.fz);
        const int a = X % g.n, ez = Z / g.n, bb = Z - ez * g.n;
        const double wq = g.wq[a] * g.wq[bb] * g.hx * g.hz[ez] * 0.25;
        s = fma(wq, u[(long long)r * u_ld + e], s);
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[(long long)r * nch + blockIdx.x] = s;
}

__global__ void __launch_bounds__(VB) gauge_apply_kernel(GridArgs g, double* __restrict__ u, long long u_ld,
                                                        const int* __restrict__ apply,
                                                        const double* __restrict__ part, int nch, int ch) {
    const int r = blockIdx.y;
    if (!apply[r]) return;
    __shared__ double red[32];
    double s = 0.0;
    for (int c = threadIdx.x; c < nch; c += VB) s += part[(long long)r * nch + c];
    s = block_sum(s, red) / g.area;
    const long long e0 = (long long)blockIdx.x * ch;
    const long long e1 = min(e0 + (long long)ch, g.r);
    for (long long e = e0 + threadIdx.x; e < e1; e += VB) u[(long long)r * u_ld + e] -= s;
}

void k_gauge(const GridArgs& g, int R, double* u, long long u_ld, const int* apply, double* part,
             int nch, int ch, cudaStream_t s) {
    dim3 grid(nch, R);
    gauge_partial_kernel<<<grid, VB, 0, s>>>(g, u, u_ld, apply, part, nch, ch);
    count_launches(1);
    gauge_apply_kernel<<<grid, VB, 0, s>>>(g, u, u_ld, apply, part, nch, ch);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Setup builders
// ---------------------------------------------------------------------------
__global__ void build_strip_op_kernel(double* __restrict__ A, const double* __restrict__ Ax,
                                      const double* __restrict__ Lz, double k2, int n, int fz) {
    const long long m = (long long)n * fz;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    const long long row = idx / m, col = idx - row * m;
    const int a = (int)(row / fz), Z = (int)(row - (long long)a * fz);
    const int ap = (int)(col / fz), Zp = (int)(col - (long long)ap * fz);
    double v = 0.0;
    if (Z == Zp) v += Ax[a * n + ap];
    if (a == ap) v += Lz[(long long)Z * fz + Zp];
    if (row == col) v -= k2;
    A[idx] = v;
}

void k_build_strip_op(double* A, const double* Ax, const double* Lz, double k2, int n, int fz,
                      cudaStream_t s) {
    const long long m = (long long)n * fz;
    const long long tot = m * m;
    build_strip_op_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A, Ax, Lz, k2, n, fz);
    count_launches(1);
}

__global__ void identity_kernel(double* X, int m) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tot = (long long)m * m;
    if (idx >= tot) return;
    const long long i = idx / m, j = idx - i * m;
    X[idx] = (i == j) ? 1.0 : 0.0;
}

void k_identity(double* X, int m, cudaStream_t s) {
    const long long tot = (long long)m * m;
    identity_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, m);
    count_launches(1);
}

// done[r] = !active[r]: the inner solve of the nested mixed-precision form runs
// only for the right-hand sides whose outer Arnoldi process is still active.
__global__ void invert_flags_kernel(int* __restrict__ done, const int* __restrict__ active, int R) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) done[r] = active[r] ? 0 : 1;
}

void k_invert_flags(int* done, const int* active, int R, cudaStream_t s) {
    invert_flags_kernel<<<(R + 127) / 128, 128, 0, s>>>(done, active, R);
    count_launches(1);
}

// Coarse division of the singular coarse matrix (Sec. 3.3): K = A^-1 (I - u u^T)
// = A^-1 - (A^-1 u) u^T in place on the row-major d x d buffer holding A^-1.
// w = A^-1 u: one warp per row.
__global__ void rowdot_kernel(double* __restrict__ w, const double* __restrict__ A, const double* __restrict__ u, int d) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= d) return;
    const double* a = A + (size_t)row * d;
    double acc = 0.0;
    for (int j = lane; j < d; j += 32) acc += a[j] * u[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) w[row] = acc;
}

__global__ void rank1_sub_kernel(double* __restrict__ A, const double* __restrict__ w, const double* __restrict__ u, int d) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)d * d) return;
    const int i = (int)(idx / d), j = (int)(idx - (long long)i * d);
    A[idx] -= w[i] * u[j];
}

// K = T^-1 (row-major d x d) of a tridiagonal T from its pivoted LU factors
// (tridiag_lu): thread j solves T x = e_j and writes x into column j of K,
// which also holds the forward-substitution values in between.  The threads
// of a warp take adjacent columns, so every row access is one coalesced line.
// fac: [dl (d-1)][dd (d)][du (d-1)][du2 (d-2)], swap: [d-1].
__global__ void tridiag_inverse_kernel(double* __restrict__ K, const double* __restrict__ fac,
                                       const int* __restrict__ swap, int d) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    const double* dl = fac;
    const double* dd = dl + (d - 1);
    const double* du = dd + d;
    const double* du2 = du + (d - 1);
    // forward: L y = P e_j (rows above j - 1 stay zero: the interchanges
    // before step j - 1 only mix zeros)
    for (int i = 0; i < j - 1; ++i) K[(long long)i * d + j] = 0.0;
    const int i0 = j > 0 ? j - 1 : 0;
    double cur = (i0 == j) ? 1.0 : 0.0;            // y[i] at step i
    for (int i = i0; i + 1 < d; ++i) {
        const double nxt = (i + 1 == j) ? 1.0 : 0.0;   // untouched entry i+1 of e_j
        double yi, yn;
        if (swap[i]) {
            yi = nxt;
            yn = cur - dl[i] * nxt;
        } else {
            yi = cur;
            yn = nxt - dl[i] * cur;
        }
        K[(long long)i * d + j] = yi;
        cur = yn;
    }
    // backward: U x = y, U with two superdiagonals
    double x1 = cur / dd[d - 1], x2 = 0.0;         // x[i+1], x[i+2]
    K[(long long)(d - 1) * d + j] = x1;
    for (int i = d - 2; i >= 0; --i) {
        double v = K[(long long)i * d + j] - du[i] * x1;
        if (i + 2 < d) v -= du2[i] * x2;
        v /= dd[i];
        K[(long long)i * d + j] = v;
        x2 = x1;
        x1 = v;
    }
}

void k_tridiag_inverse(double* K, const double* fac, const int* swap, int d, cudaStream_t s) {
    tridiag_inverse_kernel<<<(d + 127) / 128, 128, 0, s>>>(K, fac, swap, d);
    count_launches(1);
}

void k_project_coarse(double* K, double* w, const double* u, int d, cudaStream_t s) {
    rowdot_kernel<<<(d + 7) / 8, 256, 0, s>>>(w, K, u, d);
    const long long tot = (long long)d * d;
    rank1_sub_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(K, w, u, d);
    count_launches(2);
}

// W = B_c A_c^-1 (2 fz x n fz): row (s, Z) = sum_a beta[s][a] Ainv[(a, Z), :]
__global__ void build_W_kernel(double* __restrict__ W, const double* __restrict__ Ainv,
                               const double* __restrict__ beta, int n, int fz) {
    const long long m = (long long)n * fz;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2LL * fz * m) return;
    const long long row = idx / m, col = idx - row * m;
    const int s = (int)(row / fz), Z = (int)(row - (long long)s * fz);
    double v = 0.0;
    for (int a = 0; a < n; ++a) v = fma(beta[s * n + a], Ainv[((long long)a * fz + Z) * m + col], v);
    W[idx] = v;
}

void k_build_W(double* W, const double* Ainv, const double* beta, int n, int fz, cudaStream_t s) {
    const long long tot = 2LL * fz * n * fz;
    build_W_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(W, Ainv, beta, n, fz);
    count_launches(1);
}

// G = W E_c (2 fz x 2 fz): columns of W at the strip's west (a = 0) and east
// (a = N) face nodes; the physical face of a boundary class is zeroed.
__global__ void build_G_kernel(double* __restrict__ G, const double* __restrict__ W, int n, int fz, int cls) {
    const long long m = (long long)n * fz;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * fz * fz) return;
    const int row = idx / (2 * fz), col = idx - row * 2 * fz;
    const int sp = col / fz, Zp = col - sp * fz;
    const int a = sp == 0 ? 0 : n - 1;
    double v = W[(long long)row * m + (long long)a * fz + Zp];
    if ((cls == 0 && sp == 0) || (cls == 2 && sp == 1)) v = 0.0;
    G[idx] = v;
}

void k_build_G(double* G, const double* W, int n, int fz, int cls, cudaStream_t s) {
    const int tot = 4 * fz * fz;
    build_G_kernel<<<(tot + 255) / 256, 256, 0, s>>>(G, W, n, fz, cls);
    count_launches(1);
}

// Block-Jacobi block (Sec. 3.2).  Full pair, local faces 0..3 = (east face of
// strip 2p, west and east faces of strip 2p+1, west face of strip 2p+2):
//   M = I + [0 Gb_tl Gb_tr 0; Ga_br 0 0 0; 0 0 0 Gc_tl; 0 Gb_bl Gb_br 0]
// with G?_xy the (out half x, in face y) block of that strip's G.  Single
// interface (gC == null), local faces (east of 2p, west of 2p+1):
//   M = I + [0 Gb_tl; Ga_br 0].
__global__ void build_M_kernel(double* __restrict__ M, const double* __restrict__ gA, const double* __restrict__ gB,
                               const double* __restrict__ gC, int fz) {
    const int nb = gC ? 4 : 2;
    const int m = nb * fz;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    const int row = idx / m, col = idx - row * m;
    const int bi = row / fz, zi = row - bi * fz, bj = col / fz, zj = col - bj * fz;
    const int f2 = 2 * fz;
    auto gblk = [&](const double* G, int outh, int inf) { return G[(outh * fz + zi) * f2 + inf * fz + zj]; };
    double v = (row == col) ? 1.0 : 0.0;
    if (nb == 4) {
        if (bi == 0 && bj == 1) v += gblk(gB, 0, 0);
        if (bi == 0 && bj == 2) v += gblk(gB, 0, 1);
        if (bi == 3 && bj == 1) v += gblk(gB, 1, 0);
        if (bi == 3 && bj == 2) v += gblk(gB, 1, 1);
        if (bi == 1 && bj == 0) v += gblk(gA, 1, 1);
        if (bi == 2 && bj == 3) v += gblk(gC, 0, 0);
    } else {
        if (bi == 1 && bj == 0) v += gblk(gA, 1, 1);
        if (bi == 0 && bj == 1) v += gblk(gB, 0, 0);
    }
    M[idx] = v;
}

void k_build_M(double* M, const double* gA, const double* gB, const double* gC, int fz, cudaStream_t s) {
    const int m = (gC ? 4 : 2) * fz;
    build_M_kernel<<<(m * m + 255) / 256, 256, 0, s>>>(M, gA, gB, gC, fz);
    count_launches(1);
}

__global__ void pad_block_kernel(double* __restrict__ dst, const double* __restrict__ src, int ms, int md) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= md * md) return;
    const int i = idx / md, j = idx - i * md;
    dst[idx] = (i < ms && j < ms) ? src[i * ms + j] : 0.0;
}

void k_pad_block(double* dst, const double* src, int m_src, int m_dst, cudaStream_t s) {
    pad_block_kernel<<<(m_dst * m_dst + 255) / 256, 256, 0, s>>>(dst, src, m_src, m_dst);
    count_launches(1);
}

// rho[side][g][row] = sum over group g of the side's input face of G[row][.]
__global__ void build_rho_kernel(double* __restrict__ rho, const double* __restrict__ G, int fz, int ng) {
    const int f2 = 2 * fz;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * ng * f2) return;
    const int row = idx % f2, sg = idx / f2, g = sg % ng, side = sg / ng;
    const int gs = fz / ng;
    double v = 0.0;
    for (int z = 0; z < gs; ++z) v += G[row * f2 + side * fz + g * gs + z];
    rho[idx] = v;
}

void k_build_rho(double* rho, const double* G, int fz, int ng, cudaStream_t s) {
    const int tot = 2 * ng * 2 * fz;
    build_rho_kernel<<<(tot + 255) / 256, 256, 0, s>>>(rho, G, fz, ng);
    count_launches(1);
}

__global__ void fill_kernel(double* x, long long n, double v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__global__ void to_fp32_kernel(float* dst, const double* src, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (float)src[i];
}

__global__ void identity_f_kernel(float* X, int m) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m * m) return;
    const long long i = idx / m, j = idx - i * m;
    X[idx] = (i == j) ? 1.0f : 0.0f;
}

void k_identity_f(float* X, int m, cudaStream_t s) {
    const long long tot = (long long)m * m;
    identity_f_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, m);
    count_launches(1);
}

__global__ void pad_block_f_kernel(float* __restrict__ dst, const float* __restrict__ src, int ms, int md) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= md * md) return;
    const int i = idx / md, j = idx - i * md;
    dst[idx] = (i < ms && j < ms) ? src[i * ms + j] : 0.0f;
}

void k_pad_block_f(float* dst, const float* src, int m_src, int m_dst, cudaStream_t s) {
    pad_block_f_kernel<<<(m_dst * m_dst + 255) / 256, 256, 0, s>>>(dst, src, m_src, m_dst);
    count_launches(1);
}

void k_to_fp32(float* dst, const double* src, long long n, cudaStream_t s) {
    if (n <= 0) return;
    to_fp32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(dst, src, n);
    count_launches(1);
}

void k_fill(double* x, long long n, double v, cudaStream_t s) {
    if (n <= 0) return;
    fill_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, v);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// Fast strip solver: A_c(k)^-1 = (Q_c (x) I) (B_c (+) L_z - k^2)^-1 (Q_c^-1 (x) I)
// with Ax_c = Q_c B_c Q_c^-1 (real block form).  The x-transforms below apply
// an n x n class matrix along every x-line of every strip; the block solves
// are class GEMMs over the slots of B_c.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(VB) xform_kernel(FssArgs f, const double* __restrict__ T, const double* __restrict__ in,
                                                  long long in_ld, double* __restrict__ out, long long out_ld,
                                                  const double* __restrict__ xS, long long x_ld,
                                                  const double* __restrict__ addv, long long add_ld) {
    extern __shared__ double Ts[];                       // [3][n][n]
    const int n = f.n, fz = f.fz;
    for (int i = threadIdx.x; i < 3 * n * n; i += VB) Ts[i] = T[i];
    __syncthreads();
    const int r = blockIdx.y;
    const long long line = (long long)blockIdx.x * VB + threadIdx.x;   // strip * fz + Z
    if (line >= (long long)f.nstrips * fz) return;
    const int strip = (int)(line / fz), Z = (int)(line - (long long)strip * fz);
    const double* Tc = Ts + f.cls[strip] * n * n;
    const double* src = in + (long long)r * in_ld + (long long)strip * n * fz + Z;
    double u[33];
#pragma unroll 4
    for (int b = 0; b < n; ++b) u[b] = src[(long long)b * fz];
    if (xS) {   // recovery input b - E x_S: x_S on the strip's west (a = 0) and east (a = N) faces
        const double* x = xS + (long long)r * x_ld;
        u[0] -= x[(long long)(2 * strip) * fz + Z];
        u[n - 1] -= x[(long long)(2 * strip + 1) * fz + Z];
    }
    double* dst = out + (long long)r * out_ld + (long long)strip * n * fz + Z;
    const double* ad = addv ? addv + (long long)r * add_ld + (long long)strip * n * fz + Z : nullptr;
    for (int a = 0; a < n; ++a) {
        double s = ad ? ad[(long long)a * fz] : 0.0;
        for (int b = 0; b < n; ++b) s = fma(Tc[a * n + b], u[b], s);
        dst[(long long)a * fz] = s;
    }
}

void k_xform(const FssArgs& f, int R, const double* T, const double* in, long long in_ld, double* out,
             long long out_ld, const double* xS, long long x_ld, cudaStream_t s, const double* addv, long long add_ld) {
    dim3 grid((unsigned)(((long long)f.nstrips * f.fz + VB - 1) / VB), R);
    xform_kernel<<<grid, VB, (size_t)3 * f.n * f.n * sizeof(double), s>>>(f, T, in, in_ld, out, out_ld, xS, x_ld,
                                                                            addv, add_ld);
    count_launches(1);
}

// Residual of the strip systems in FP64: res = (b - E x_S) - A_c(k) x with
// A_c(k) = Ax_c (+) L_z - k^2 applied through its Kronecker-sum structure
// (n + |window| FMAs per node: L_z row Z is nonzero only on [zlo[Z], zhi[Z])).
__global__ void __launch_bounds__(VB) strip_residual_kernel(FssArgs f, const double* __restrict__ Ax3,
                                                           const double* __restrict__ Lz, const int* __restrict__ zlo,
                                                           const int* __restrict__ zhi, const double* __restrict__ k2r,
                                                           const double* __restrict__ b, long long b_ld,
                                                           const double* __restrict__ xS, long long x_ld,
                                                           const double* __restrict__ x, long long xv_ld,
                                                           double* __restrict__ res, long long r_ld) {
    const int r = blockIdx.y;
    const int n = f.n, fz = f.fz;
    const long long node = (long long)blockIdx.x * VB + threadIdx.x;
    const long long per = (long long)n * fz;
    if (node >= (long long)f.nstrips * per) return;
    const int strip = (int)(node / per);
    const int rem = (int)(node - (long long)strip * per);
    const int a = rem / fz, Z = rem - a * fz;
    const double* xs = x + (long long)r * xv_ld + (long long)strip * per;
    const double* Axc = Ax3 + (long long)f.cls[strip] * n * n + a * n;
    double ax = 0.0;
    for (int bb = 0; bb < n; ++bb) ax = fma(Axc[bb], xs[(long long)bb * fz + Z], ax);
    const double* lz = Lz + (long long)Z * fz;
    const double* xa = xs + (long long)a * fz;
    for (int zz = zlo[Z]; zz < zhi[Z]; ++zz) ax = fma(lz[zz], xa[zz], ax);
    ax -= k2r[r] * xa[Z];
    double bv = b[(long long)r * b_ld + node];
    if (xS) {
        const double* xsr = xS + (long long)r * x_ld;
        if (a == 0) bv -= xsr[(long long)(2 * strip) * fz + Z];
        if (a == n - 1) bv -= xsr[(long long)(2 * strip + 1) * fz + Z];
    }
    res[(long long)r * r_ld + node] = bv - ax;
}

void k_strip_residual(const FssArgs& f, int R, const double* Ax3, const double* Lz, const int* zlo, const int* zhi,
                      const double* k2r, const double* b, long long b_ld, const double* xS, long long x_ld,
                      const double* x, long long xv_ld, double* res, long long r_ld, cudaStream_t s) {
    const long long tot = (long long)f.nstrips * f.n * f.fz;
    dim3 grid((unsigned)((tot + VB - 1) / VB), R);
    strip_residual_kernel<<<grid, VB, 0, s>>>(f, Ax3, Lz, zlo, zhi, k2r, b, b_ld, xS, x_ld, x, xv_ld, res, r_ld);
    count_launches(1);
}

// b_S = B y: face (strip i, side s) receives -tau (u +- d/dx u) of the neighbour
// strip's solution y at the coincident face, i.e. sum_a beta_c[.][a] y[a][Z].
__global__ void __launch_bounds__(VB) face_flux_kernel(FssArgs f, const double* __restrict__ beta,
                                                      const double* __restrict__ y, long long y_ld,
                                                      double* __restrict__ bS, long long b_ld, long long kp) {
    const int r = blockIdx.y;
    const long long e = (long long)blockIdx.x * VB + threadIdx.x;
    if (e >= kp) return;
    const int n = f.n, fz = f.fz;
    const int F = (int)(e / fz), Z = (int)(e - (long long)F * fz);
    const int i = F >> 1, side = F & 1;
    double v = 0.0;
    if (F > 0 && F < 2 * f.nstrips - 1) {
        const int src = side == 1 ? i + 1 : i - 1;      // neighbour strip
        const int sel = side == 1 ? 0 : 1;              // its flux onto its west / east neighbour
        const double* bt = beta + (f.cls[src] * 2 + sel) * n;
        const double* ys = y + (long long)r * y_ld + (long long)src * n * fz + Z;
        for (int a = 0; a < n; ++a) v = fma(bt[a], ys[(long long)a * fz], v);
    }
    bS[(long long)r * b_ld + e] = v;
}

void k_face_flux(const FssArgs& f, int R, const double* beta, const double* y, long long y_ld, double* bS,
                 long long b_ld, long long kp, cudaStream_t s) {
    dim3 grid((unsigned)((kp + VB - 1) / VB), R);
    face_flux_kernel<<<grid, VB, 0, s>>>(f, beta, y, y_ld, bS, b_ld, kp);
    count_launches(1);
}

// Slot matrix of B_c (+) L_z - k^2: size 1: L_z + (alpha - k^2) I (fz x fz);
// size 2: [[L_z + (alpha - k^2) I, beta I], [-beta I, L_z + (alpha - k^2) I]].
__global__ void build_slot_kernel(double* __restrict__ M, const double* __restrict__ Lz, int fz, int size,
                                  double shift, double beta) {
    const int m = size * fz;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m * m) return;
    const int row = (int)(idx / m), col = (int)(idx - (long long)row * m);
    const int bi = row / fz, zi = row - bi * fz, bj = col / fz, zj = col - bj * fz;
    double v = 0.0;
    if (bi == bj) v = Lz[(long long)zi * fz + zj] + (zi == zj ? shift : 0.0);
    else if (zi == zj) v = (bi == 0) ? beta : -beta;
    M[idx] = v;
}

void k_build_slot(double* M, const double* Lz, int fz, int size, double shift, double beta, cudaStream_t s) {
    const long long tot = (long long)size * fz * size * fz;
    build_slot_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(M, Lz, fz, size, shift, beta);
    count_launches(1);
}

// Batched inversion by Gauss-Jordan elimination with partial pivoting, one
// CTA per matrix (row-major n x n): the pivot row is scaled in place with its
// pivot entry replaced by 1 (so that column k of the other rows becomes the
// inverse's column), every other row is eliminated, and the column order is
// restored at the end by undoing the row interchanges in reverse.  SM: the
// working matrix in shared memory (n <= kGjSmemMax), else in dst (global
// memory, L2-resident while the CTA works on it).  info[b] = k + 1 if the
// pivot of step k is zero or not finite (dst then holds no inverse).
constexpr int GJ_THREADS = 256;

template <bool SM>
__global__ void __launch_bounds__(GJ_THREADS) gj_inverse_kernel(const double* const* __restrict__ src,
                                                               double* const* __restrict__ dst, int n,
                                                               int* __restrict__ info) {
    extern __shared__ double gj_sh[];
    __shared__ double red_v[GJ_THREADS / 32];
    __shared__ int red_i[GJ_THREADS / 32];
    __shared__ int s_p, s_fail;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = GJ_THREADS / 32;
    double* W = SM ? gj_sh : dst[b];
    double* col = SM ? gj_sh + (size_t)n * n : gj_sh;
    int* piv = reinterpret_cast<int*>(col + n);
    const double* S = src[b];
    for (long long idx = tid; idx < (long long)n * n; idx += GJ_THREADS) W[idx] = S[idx];
    if (tid == 0) s_fail = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        // pivot: the largest |W[i][k]|, i >= k (smallest i among equals)
        double best = -1.0;
        int bi = n;
        for (int i = k + tid; i < n; i += GJ_THREADS) {
            const double v = fabs(W[(long long)i * n + k]);
            if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { red_v[warp] = best; red_i[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            double bv = red_v[0];
            int bx = red_i[0];
            for (int w = 1; w < NW; ++w)
                if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bx)) { bv = red_v[w]; bx = red_i[w]; }
            s_p = bx;
            if (!(bv > 0.0) || !isfinite(bv) || bx >= n) s_fail = k + 1;
        }
        __syncthreads();
        if (s_fail) break;
        const int p = s_p;
        if (tid == 0) piv[k] = p;
        if (p != k)
            for (int j = tid; j < n; j += GJ_THREADS) {
                const double t = W[(long long)k * n + j];
                W[(long long)k * n + j] = W[(long long)p * n + j];
                W[(long long)p * n + j] = t;
            }
        __syncthreads();
        const double pinv = 1.0 / W[(long long)k * n + k];
        for (int i = tid; i < n; i += GJ_THREADS) col[i] = W[(long long)i * n + k];
        __syncthreads();
        for (int j = tid; j < n; j += GJ_THREADS)
            W[(long long)k * n + j] = (j == k ? 1.0 : W[(long long)k * n + j]) * pinv;
        __syncthreads();
        for (int i = warp; i < n; i += NW) {
            if (i == k) continue;
            const double f = col[i];
            double* Wi = W + (long long)i * n;
            const double* Wk = W + (long long)k * n;
            for (int j = lane; j < n; j += 32) Wi[j] = (j == k) ? -Wk[k] * f : fma(-Wk[j], f, Wi[j]);
        }
        __syncthreads();
    }
    if (!s_fail) {
        for (int k = n - 1; k >= 0; --k) {
            const int p = piv[k];
            if (p != k)
                for (int i = tid; i < n; i += GJ_THREADS) {
                    const double t = W[(long long)i * n + k];
                    W[(long long)i * n + k] = W[(long long)i * n + p];
                    W[(long long)i * n + p] = t;
                }
            __syncthreads();
        }
        if (SM) {
            double* D = dst[b];
            for (long long idx = tid; idx < (long long)n * n; idx += GJ_THREADS) D[idx] = W[idx];
        }
    }
    if (tid == 0) info[b] = s_fail;
}

int gj_smem_max() { return 158; }

void k_gj_inverse(const double* const* src, double* const* dst, int n, int count, int* info, cudaStream_t s) {
    if (count <= 0) return;
    const auto smem_of = [](int m) {
        return (size_t)m * m * sizeof(double) + (size_t)m * sizeof(double) + (size_t)m * sizeof(int);
    };
    if (n <= gj_smem_max()) {
        static std::once_flag once;   // setups on several host threads
        std::call_once(once, [&] {
            cudaFuncSetAttribute(gj_inverse_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_of(gj_smem_max()));
        });
        gj_inverse_kernel<true><<<count, GJ_THREADS, smem_of(n), s>>>(src, dst, n, info);
    } else {
        const size_t sh = (size_t)n * sizeof(double) + (size_t)n * sizeof(int);
        gj_inverse_kernel<false><<<count, GJ_THREADS, sh, s>>>(src, dst, n, info);
    }
    count_launches(1);
}

// The two half-size matrices of a reversal-symmetric slot matrix M (uniform
// h_z): with p the first half of the z-nodes of each f_z block and q = J p
// their mirror images, M = [[A, B], [B, A]] in (p, q) order and
// M^-1 = the mirror form with halves (A + B)^-1 / 2 and (A - B)^-1 / 2.
// Writes 2 (A + B) at H and 2 (A - B) at H + h^2 (h = size fz / 2, row-major),
// whose inverses are those halves.
__global__ void build_slot_halves_kernel(double* __restrict__ H, const double* __restrict__ Lz, int fz, int size,
                                         double shift, double beta) {
    const int hb = fz / 2, h = size * hb;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)h * h) return;
    const int i = (int)(idx / h), j = (int)(idx - (long long)i * h);
    const int bi = i / hb, zi = i - bi * hb;              // row p(i): block bi, node zi
    const int bj = j / hb, zp = j - bj * hb, zq = fz - 1 - zp;   // columns p(j), q(j) in block bj
    double vp = 0.0, vq = 0.0;
    if (bi == bj) {
        vp = Lz[(long long)zi * fz + zp] + (zi == zp ? shift : 0.0);
        vq = Lz[(long long)zi * fz + zq] + (zi == zq ? shift : 0.0);
    } else {
        const double b = bi == 0 ? beta : -beta;
        vp = zi == zp ? b : 0.0;
        vq = zi == zq ? b : 0.0;
    }
    H[idx] = 2.0 * (vp + vq);
    H[(long long)h * h + idx] = 2.0 * (vp - vq);
}

void k_build_slot_halves(double* H, const double* Lz, int fz, int size, double shift, double beta, cudaStream_t s) {
    const long long h = (long long)size * fz / 2, tot = h * h;
    build_slot_halves_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(H, Lz, fz, size, shift, beta);
    count_launches(1);
}

// Unit right-hand sides for the Schur blocks: column j < fz is the west-face
// node (a = 0, Z = j) of one strip, column j >= fz the east-face node (a = N).
__global__ void unit_faces_kernel(double* __restrict__ U, int n, int fz) {
    const long long nfz = (long long)n * fz;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2LL * fz * nfz) return;
    const int j = (int)(idx / nfz);
    const long long p = idx - (long long)j * nfz;
    const long long hot = j < fz ? (long long)j : (long long)(n - 1) * fz + (j - fz);
    U[idx] = (p == hot) ? 1.0 : 0.0;
}

void k_unit_faces(double* U, int n, int fz, cudaStream_t s) {
    const long long tot = 2LL * fz * n * fz;
    unit_faces_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(U, n, fz);
    count_launches(1);
}

// G_c[(s, Z)][j] = sum_a beta_c[s][a] Y_j[a][Z] (Y_j = A_c^-1 of unit column j);
// the physical face's columns of a boundary class are zero.
__global__ void g_from_solves_kernel(double* __restrict__ G, const double* __restrict__ Y, const double* __restrict__ beta,
                                     int n, int fz, int cls) {
    const int f2 = 2 * fz;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= f2 * f2) return;
    const int row = idx / f2, j = idx - row * f2;
    const int s = row / fz, Z = row - s * fz;
    const double* y = Y + (long long)j * n * fz + Z;
    double v = 0.0;
    for (int a = 0; a < n; ++a) v = fma(beta[s * n + a], y[(long long)a * fz], v);
    if ((cls == 0 && j < fz) || (cls == 2 && j >= fz)) v = 0.0;
    G[idx] = v;
}

// Quality of the FP32 block-Jacobi copies: for each m x m block (row-major,
// FP64 inverse A and its FP32 copy B), the relative difference
// |A v - B v| / |A v| of the FP64 product and the FP32 product (FP32 inputs and
// accumulation, as the mixed apply does) for a fixed sign vector v.  One block
// of VB threads per matrix; out[i] receives the ratio.
__global__ void __launch_bounds__(VB) fp32_quality_kernel(const double* __restrict__ A, const float* __restrict__ B,
                                                         int m, long long stride, double* __restrict__ out) {
    __shared__ double red[32];
    const double* a = A + (long long)blockIdx.x * stride;
    const float* b = B + (long long)blockIdx.x * stride;
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < m; i += VB) {
        double y64 = 0.0;
        float y32 = 0.0f;
        for (int j = 0; j < m; ++j) {
            const unsigned hsh = (unsigned)j * 2654435761u;
            const double v = (hsh & 0x10000u) ? 1.0 : -1.0;
            y64 = fma(a[(long long)i * m + j], v, y64);
            y32 = fmaf(b[(long long)i * m + j], (float)v, y32);
        }
        num = fma(y64 - (double)y32, y64 - (double)y32, num);
        den = fma(y64, y64, den);
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    if (threadIdx.x == 0) out[blockIdx.x] = den > 0.0 ? sqrt(num / den) : 0.0;
}

void k_fp32_quality(const double* A, const float* B, int m, long long stride, int nmat, double* out, cudaStream_t s) {
    fp32_quality_kernel<<<nmat, VB, 0, s>>>(A, B, m, stride, out);
    count_launches(1);
}

// Real DFT along y (Sec. 5, Eq. fourier_poisson) for the physical-space 3-D
// solve.  in: [my][n] samples at y_t = t l_y / my; out: [my/2+1][2][n] with
// u(y) = sum_j u_j e^{i k_j y}: u_j = (1/my) sum_t u(y_t) e^{-2 pi i j t / my}.
// cs: [2][my] table of cos and sin of 2 pi idx / my.
static constexpr int DFT_W = 4;   // modes (forward) or planes (inverse) per thread: each load serves four

__global__ void __launch_bounds__(VB) dft_forward_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                        const double* __restrict__ cs, long long n, int my) {
    extern __shared__ double tab[];
    for (int i = threadIdx.x; i < 2 * my; i += VB) tab[i] = cs[i];
    __syncthreads();
    const int h = my / 2;
    const int j0 = blockIdx.y * DFT_W;
    const long long i = (long long)blockIdx.x * VB + threadIdx.x;
    if (i >= n) return;
    // samples t and my - t share cos(2 pi j t / my) and carry opposite sines:
    // re_j = v_0 + (-1)^j v_{my/2} + sum_{0<t<my/2} (v_t + v_{my-t}) cos,
    // im_j = -sum_{0<t<my/2} (v_t - v_{my-t}) sin
    const double v0 = in[i], vh = in[(long long)h * n + i];
    double re[DFT_W], im[DFT_W];
    int idx[DFT_W];                                // (j t) mod my, stepped
#pragma unroll
    for (int w = 0; w < DFT_W; ++w) {
        re[w] = v0 + (((j0 + w) & 1) ? -vh : vh);
        im[w] = 0.0;
        idx[w] = (j0 + w) % my;
    }
    for (int t = 1; t < h; ++t) {
        const double a = in[(long long)t * n + i], b = in[(long long)(my - t) * n + i];
        const double sp = a + b, sm = b - a;
#pragma unroll
        for (int w = 0; w < DFT_W; ++w) {
            re[w] = fma(sp, tab[idx[w]], re[w]);
            im[w] = fma(sm, tab[my + idx[w]], im[w]);
            idx[w] += j0 + w;
            if (idx[w] >= my) idx[w] -= my;
        }
    }
    const double inv = 1.0 / my;
#pragma unroll
    for (int w = 0; w < DFT_W; ++w) {
        const int j = j0 + w;
        if (j > h) break;
        out[(long long)(2 * j) * n + i] = re[w] * inv;
        out[(long long)(2 * j + 1) * n + i] = (j == 0 || j == h) ? 0.0 : im[w] * inv;
    }
}

// Inverse: u(y_t) = Re u_0 + Re u_{my/2} (-1)^t + 2 sum_{0<j<my/2} Re(u_j e^{2 pi i j t / my});
// outputs t and my - t together (same cosines, opposite sines), t in [0, my/2]
__global__ void __launch_bounds__(VB) dft_inverse_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                        const double* __restrict__ cs, long long n, int my) {
    extern __shared__ double tab[];
    for (int i = threadIdx.x; i < 2 * my; i += VB) tab[i] = cs[i];
    __syncthreads();
    const int h = my / 2;
    const int t0 = blockIdx.y * DFT_W;
    const long long i = (long long)blockIdx.x * VB + threadIdx.x;
    if (i >= n) return;
    const double u0 = in[i], uh = in[(long long)(2 * h) * n + i];
    double A[DFT_W], B[DFT_W];
    int idx[DFT_W];                                // (j t) mod my, stepped
#pragma unroll
    for (int w = 0; w < DFT_W; ++w) {
        A[w] = u0 + (((t0 + w) & 1) ? -uh : uh);
        B[w] = 0.0;
        idx[w] = (t0 + w) % my;
    }
    for (int j = 1; j < h; ++j) {
        const double re = 2.0 * in[(long long)(2 * j) * n + i], im = 2.0 * in[(long long)(2 * j + 1) * n + i];
#pragma unroll
        for (int w = 0; w < DFT_W; ++w) {
            A[w] = fma(re, tab[idx[w]], A[w]);
            B[w] = fma(im, tab[my + idx[w]], B[w]);
            idx[w] += t0 + w;
            if (idx[w] >= my) idx[w] -= my;
        }
    }
#pragma unroll
    for (int w = 0; w < DFT_W; ++w) {
        const int t = t0 + w;
        if (t > h) break;
        out[(long long)t * n + i] = A[w] - B[w];
        if (t != 0 && t != h) out[(long long)(my - t) * n + i] = A[w] + B[w];
    }
}

void k_dft_forward(const double* in, double* out, const double* cs, long long n, int my, cudaStream_t s) {
    dim3 grid((unsigned)((n + VB - 1) / VB), (my / 2 + 1 + DFT_W - 1) / DFT_W);
    dft_forward_kernel<<<grid, VB, (size_t)2 * my * sizeof(double), s>>>(in, out, cs, n, my);
    count_launches(1);
}

void k_dft_inverse(const double* in, double* out, const double* cs, long long n, int my, cudaStream_t s) {
    dim3 grid((unsigned)((n + VB - 1) / VB), (my / 2 + 1 + DFT_W - 1) / DFT_W);
    dft_inverse_kernel<<<grid, VB, (size_t)2 * my * sizeof(double), s>>>(in, out, cs, n, my);
    count_launches(1);
}

// dst = P src P for an (nb fz) x (nb fz) row-major matrix, P reversing the
// order of its nb face blocks (z order inside a block kept): the operator of
// the mirror-image strip or strip pair (x -> -x swaps east and west faces).
__global__ void mirror_blocks_kernel(double* __restrict__ dst, const double* __restrict__ src, int fz, int nb) {
    const long long m = (long long)nb * fz;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    const long long i = idx / m, j = idx - i * m;
    const long long pi = (nb - 1 - i / fz) * fz + i % fz, pj = (nb - 1 - j / fz) * fz + j % fz;
    dst[idx] = src[pi * m + pj];
}

void k_mirror_blocks(double* dst, const double* src, int fz, int nb, cudaStream_t s) {
    const long long tot = (long long)nb * fz * nb * fz;
    mirror_blocks_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(dst, src, fz, nb);
    count_launches(1);
}

// mirror(i) over the full column of nb faces
__device__ __forceinline__ long long mirror_full(long long i, int fz, int nb) {
    return (nb - 1 - i / fz) * fz + i % fz;
}

__global__ void mirror_asym_kernel(const double* __restrict__ Mat, int fz, int nb, double* res) {
    __shared__ double sh[2][32];
    const long long m = (long long)nb * fz;
    double dmax = 0.0, amax = 0.0;
    for (long long idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
        const long long i = idx / m, j = idx - i * m;
        const double v = Mat[idx];
        dmax = fmax(dmax, fabs(v - Mat[mirror_full(i, fz, nb) * m + mirror_full(j, fz, nb)]));
        amax = fmax(amax, fabs(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = dmax;
        sh[1][wid] = amax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            dmax = fmax(dmax, sh[0][w]);
            amax = fmax(amax, sh[1][w]);
        }
        res[0] = dmax;
        res[1] = amax;
    }
}

void k_mirror_asym(const double* Mat, int fz, int nb, double* res, cudaStream_t s) {
    mirror_asym_kernel<<<1, 1024, 0, s>>>(Mat, fz, nb, res);
    count_launches(1);
}

// Each element pair (idx, mirror of idx) is averaged by the thread of the
// smaller index (the two never coincide for even nb).
__global__ void mirror_symmetrize_kernel(double* __restrict__ Mat, int fz, int nb) {
    const long long m = (long long)nb * fz;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    const long long i = idx / m, j = idx - i * m;
    const long long p = mirror_full(i, fz, nb) * m + mirror_full(j, fz, nb);
    if (p <= idx) return;
    const double v = 0.5 * (Mat[idx] + Mat[p]);
    Mat[idx] = v;
    Mat[p] = v;
}

void k_mirror_symmetrize(double* Mat, int fz, int nb, cudaStream_t s) {
    const long long tot = (long long)nb * fz * nb * fz;
    mirror_symmetrize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(Mat, fz, nb);
    count_launches(1);
}

template <typename T>
__global__ void mirror_halves_kernel(T* __restrict__ H, const T* __restrict__ Mat, int fz, int nb) {
    const long long m = (long long)nb * fz, h = m / 2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= h * h) return;
    const long long i = idx / h, j = idx - i * h;
    const T x = Mat[i * m + j], y = Mat[i * m + mirror_full(j, fz, nb)];
    H[idx] = T(0.5) * (x + y);
    H[h * h + idx] = T(0.5) * (x - y);
}

void k_mirror_halves(double* H, const double* Mat, int fz, int nb, cudaStream_t s) {
    const long long h = (long long)nb * fz / 2;
    mirror_halves_kernel<double><<<(unsigned)((h * h + 255) / 256), 256, 0, s>>>(H, Mat, fz, nb);
    count_launches(1);
}

void k_mirror_halves_f(float* H, const float* Mat, int fz, int nb, cudaStream_t s) {
    const long long h = (long long)nb * fz / 2;
    mirror_halves_kernel<float><<<(unsigned)((h * h + 255) / 256), 256, 0, s>>>(H, Mat, fz, nb);
    count_launches(1);
}

void k_g_from_solves(double* G, const double* Y, const double* beta, int n, int fz, int cls, cudaStream_t s) {
    const int tot = 4 * fz * fz;
    g_from_solves_kernel<<<(tot + 255) / 256, 256, 0, s>>>(G, Y, beta, n, fz, cls);
    count_launches(1);
}

// ---------------------------------------------------------------------------
// FP64 DFMA throughput probe (eight independent FMA chains per thread)
// ---------------------------------------------------------------------------
__global__ void fp64_probe_kernel(double* out, int iters) {
    double x[8];
    const double y = 0.999999, z = 1e-7;
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], y, z);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 12345.678) out[blockIdx.x] = s;  // practically never taken; keeps the chains live
}

void k_fp64_probe(double* out, int blocks, int iters, cudaStream_t s) {
    fp64_probe_kernel<<<blocks, 256, 0, s>>>(out, iters);
    count_launches(1);
}

}  // namespace smpm

// FP64-accurate dense products on the tensor cores (tcgen05, sm_103a) by
// exact integer slicing (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump 2012;
// on integer-exact tensor products: Ootomo, Ozaki & Yokota 2024).
//
// The class GEMMs of the solve (Schur products S x, block-Jacobi applies
// M^-1 x: Secs. 3.1-3.2) multiply one FP64 class matrix A (M x K) by many
// FP64 columns B.  GB300's FP64 rate is ~1.25 TFLOP/s; its BF16 tensor rate
// is ~2.25 PFLOP/s.  Each value is written as a sum of S signed integer
// digits of beta bits scaled by a power of two shared by its row of A or its
// column of B:
//     a_ik = 2^(Ea_i - S beta) X_ik,   X_ik = sum_s alpha_s 2^((S-s) beta),
//     b_kj = 2^(Eb_j - S beta) Y_kj,   Y_kj = sum_t gamma_t 2^((S-t) beta),
// |alpha|, |gamma| < 2^beta <= 128, so every digit is exact in BF16 and
// every digit product exact in FP32.  The products of the digit matrices
// are accumulated per anti-diagonal d = s + t in FP32 tensor memory,
//     D_d = sum_{s+t=d} sum_k alpha_s,ik gamma_t,kj,
// which stays an exact integer while S K (2^beta - 1)^2 < 2^24 (beta is
// chosen per K so that it does).  Keeping the diagonals d <= S + 1 drops
// terms below 2^-(S beta) of |a|_max,row |b|_max,col per product term (S beta
// >= 56 bits: at or below FP64 rounding; S beta >= 24 bits in the variant
// that replaces FP32 products), and the sum
//     (A B)_ij = 2^(Ea_i + Eb_j - (S+1) beta) sum_d 2^((S+1-d) beta) D_d
// is formed exactly in 64-bit integers and rounded once to FP64.
//
// Kernel layout: one CTA of 256 threads per tile of N = 64 (S <= 8) or 32
// (S > 8) columns; for every 128-row tile of A: the A digit blocks (128 x
// 128 BF16, pre-split at setup, stored in the tensor cores' K-major
// core-matrix order) stream into shared memory by bulk copies, the B digits
// of the K-chunk are split from FP64 by integer operations in shared
// memory, one thread issues the tcgen05.mma instructions (M = 128, K = 16),
// and the eight warps read the S accumulators back (tcgen05.ld: a warp
// reads its 32 tensor-memory lanes, i.e. rows, for half of the columns) and
// combine them.  Every wait is limited in time (0.2 s) and in tries; a wait
// that runs out sets the error word, the CTA stops issuing work, waits
// (bounded) for its tensor-core work in flight and frees its tensor memory.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "kernels.h"

namespace smpm {

namespace {

constexpr int OZ_THREADS = 256;
constexpr int OZ_KC = 128;                      // K-chunk: one shared-memory digit block
constexpr int OZ_BLOCK = 128 * OZ_KC;           // BF16 values of one 128 x 128 digit block
constexpr long long OZ_SPIN = 1LL << 22;        // iteration limit of every wait
constexpr unsigned long long OZ_WAIT_NS = 200000000ULL;   // and its time limit (0.2 s)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, no swizzle, core matrices of 8
// rows x 16 bytes; lbo = byte step between core matrices along K, sbo =
// byte step between 8-row groups.
__device__ __forceinline__ uint64_t mat_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B (both K-major) and an
// FP32 accumulator, shape M = 128 x N.
__device__ __forceinline__ uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Wait for the phase with parity `phase` of a barrier to complete; false
// once OZ_WAIT_NS of wall time (the global timer) or OZ_SPIN tries have passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (long long it = 0; it < OZ_SPIN; ++it) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(smem_addr(bar)), "r"(phase) : "memory");
        if (ok) return true;
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > OZ_WAIT_NS) return false;
    }
    return false;
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Offset (in BF16 values) of element (row, k) of a 128 x OZ_KC digit block
// in K-major core-matrix order: core (row / 8, k / 8) at (row / 8) * 2048 +
// (k / 8) * 128 bytes, row % 8 at 16 bytes, k % 8 at 2 bytes.
__host__ __device__ __forceinline__ int blk_off(int row, int k) {
    return (row >> 3) * 1024 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

// Integer X = round(v 2^(S beta - E)) of an FP64 value with |v| < 2^E, by
// integer operations on its bits (denormal inputs count as 0); clamped to
// 2^(S beta) - 1.  Returns |X| and sets neg.
__device__ __forceinline__ unsigned long long fixed_of(double v, int E, int sb, bool& neg) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    neg = (bits >> 63) != 0;
    const int eb = (int)((bits >> 52) & 0x7FF);
    if (eb == 0) return 0ULL;
    const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
    const int sh = eb - 1075 + sb - E;
    unsigned long long x;
    if (sh >= 0) {
        x = sh < 11 ? mant << sh : ~0ULL;
    } else if (sh > -64) {
        const int r = -sh;
        x = r == 0 ? mant : (mant >> r) + ((mant >> (r - 1)) & 1ULL);
    } else {
        x = 0ULL;
    }
    const unsigned long long top = (1ULL << sb) - 1ULL;
    return x > top ? top : x;
}

// BF16 bits of the signed small integer (neg ? -d : d), 0 <= d < 256.
__device__ __forceinline__ unsigned short bf16_of_digit(unsigned d, bool neg) {
    float f = __int_as_float(0x4B000000 | (int)d) - 8388608.0f;   // exactly d
    if (neg) f = -f;
    return (unsigned short)(__float_as_uint(f) >> 16);              // low 16 bits are zero
}

// Exponent E with |v| < 2^E for the largest magnitude of a row or column
// (E of the smallest normal when the maximum is 0 or denormal).
__device__ __forceinline__ int exp_bound(double amax) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(amax);
    const int eb = (int)((bits >> 52) & 0x7FF);
    return eb == 0 ? -1021 : eb - 1022;
}

}  // namespace

// Setup: the digits of every row of nmat class matrices (row-major M x K,
// matrix m at mats + m * mat_stride) and the row exponents.  Digit s of
// (matrix m, 128-row tile mt, K-chunk kc) is one 128 x 128 block in the
// tensor cores' K-major core-matrix order at
//     dig + m * dig_stride + ((mt * kcn + kc) * S + s) * OZ_BLOCK;
// rows >= M and columns >= K are zero digits.  One warp per row.
template <typename T>
__global__ void oz_split_rows_kernel(const T* __restrict__ mats, long long mat_stride, int nmat, int M, int K,
                                     int S, int beta, int mt_n, int kcn, unsigned short* __restrict__ dig,
                                     long long dig_stride, int* __restrict__ rexp, long long rexp_stride) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int rows = mt_n * 128;
    if (warp >= nmat * rows) return;
    const int m = warp / rows, row = warp - m * rows;
    const T* a = mats + (long long)m * mat_stride + (long long)row * K;
    double amax = 0.0;
    if (row < M)
        for (int k = lane; k < K; k += 32) amax = fmax(amax, fabs((double)a[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const int E = exp_bound(amax);
    if (lane == 0) rexp[(long long)m * rexp_stride + row] = E;
    const int mt = row >> 7, r = row & 127, sb = S * beta;
    const unsigned mask = (1u << beta) - 1u;
    for (int k = lane; k < kcn * OZ_KC; k += 32) {
        bool neg = false;
        const unsigned long long x = (row < M && k < K) ? fixed_of((double)a[k], E, sb, neg) : 0ULL;
        const int kc = k / OZ_KC, kk = k - kc * OZ_KC;
        unsigned short* base = dig + (long long)m * dig_stride + (long long)((mt * kcn + kc) * S) * OZ_BLOCK;
        for (int s = 0; s < S; ++s) {
            const unsigned d = (unsigned)(x >> ((S - 1 - s) * beta)) & mask;
            base[(long long)s * OZ_BLOCK + blk_off(r, kk)] = bf16_of_digit(d, neg);
        }
    }
}

namespace {

// Shared memory of the product kernel: B digits [S][N][OZ_KC], two A digit
// buffers [128][OZ_KC], column exponents, barriers, tensor-memory address.
struct OzSmemLayout {
    int b_off, a_off, e_off, bar_off, total;
    __host__ __device__ OzSmemLayout(int S, int N) {
        b_off = 0;
        a_off = S * N * OZ_KC * 2;
        e_off = a_off + 2 * OZ_BLOCK * 2;
        bar_off = e_off + 64 * 8 + 64 * 4;          // column maxima (8 B), column exponents (4 B)
        total = bar_off + 8 * 8;
    }
};

}  // namespace

// out[:, col] = A_{tile} * in[:, col] (+ add) for the column tiles of a class
// GEMM (same tile lists, addressing and epilogues as class_gemm_kernel).
template <int S, int BETA, int N>
__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(OzArgs z, const Tile* __restrict__ tiles) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    const GemmArgs& a = z.a;
    constexpr int beta = BETA;
    const int K = a.K, M = a.M;
    const OzSmemLayout L(S, N);
    unsigned short* Bd = reinterpret_cast<unsigned short*>(oz_smem + L.b_off);
    unsigned short* Ad = reinterpret_cast<unsigned short*>(oz_smem + L.a_off);
    int* colE = reinterpret_cast<int*>(oz_smem + L.e_off + 64 * 8);
    uint64_t* bars = reinterpret_cast<uint64_t*>(oz_smem + L.bar_off);   // full[2], done[2], chunk, tmem word
    uint64_t *full = bars, *done = bars + 2, *chunk = bars + 4;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 5);
    __shared__ int fail;

    const Tile t = tiles[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ncol = t.nu * t.nr;
    if (a.active) {
        int any = 0;
        for (int c = 0; c < t.nr; ++c) any |= a.active[t.r0 + c];
        if (!any) return;
    }
    if (tid == 0) {
        for (int i = 0; i < 5; ++i) mbar_init(bars + i, 1);
        fail = 0;
        if (a.flops) {   // profile: [0] algorithmic FP64 FLOPs of the tile, [1] executed tensor FLOPs
            int cols = 0;
            for (int c = 0; c < ncol; ++c) cols += (a.active == nullptr || a.active[t.r0 + c % t.nr]) ? 1 : 0;
            const int rows = max(0, min(a.row_hi[t.mat], M) - a.row_lo[t.mat]);
            atomicAdd(a.flops, 2ULL * (unsigned long long)rows * (unsigned long long)K * (unsigned long long)cols);
            atomicAdd(a.flops + 1, (unsigned long long)z.mt_n * z.kcn * (S * (S + 1) / 2) * 2ULL * 128ULL * OZ_KC *
                                       (unsigned long long)N);
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_addr(tslot)), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // column exponents over the whole K (a column outside the tile or of an
    // inactive right-hand side is all zero digits)
    // (OZ_THREADS / N threads per column, a shuffle reduction among them)
    {
        constexpr int TPC = OZ_THREADS / N;
        const int c = tid / TPC, part = tid - c * TPC;
        const bool live = c < ncol && (a.active == nullptr || a.active[t.r0 + c % t.nr]);
        double bmax = 0.0;
        if (live) {
            const int u = t.u0 + c / t.nr, r = t.r0 + c % t.nr;
            const double* col = a.in + (long long)r * a.in_rs + (long long)u * a.in_us + a.in_off + t.off;
            for (int k = part; k < K; k += TPC) bmax = fmax(bmax, fabs(col[k]));
        }
#pragma unroll
        for (int o = TPC / 2; o > 0; o >>= 1) bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        if (part == 0) colE[c] = live ? exp_bound(bmax) : -100000;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = instr_desc(N);
    const uint64_t bdesc0 = mat_desc(smem_addr(Bd), 128, 2048);
    const int kcn = z.kcn;
    constexpr int sb = S * BETA;
    constexpr unsigned mask = (1u << BETA) - 1u;
    const unsigned short* Am = z.dig + (long long)t.mat * z.dig_stride;
    uint32_t ph_full[2] = {0u, 0u}, ph_done[2] = {0u, 0u}, ph_chunk = 0u;
    constexpr int dm = S / 2;

    for (int mt = 0; mt < z.mt_n && !fail; ++mt) {
        for (int kc = 0; kc < kcn && !fail; ++kc) {
            if (!(kcn == 1 && mt > 0)) {
                // B digits of K-chunk kc: thread -> (column, 8-wide K group)
                for (int idx = tid; idx < N * (OZ_KC / 8); idx += OZ_THREADS) {
                    const int c = idx / (OZ_KC / 8), kg = idx - c * (OZ_KC / 8);
                    const int E = colE[c];
                    unsigned long long x[8];
                    bool neg[8];
                    const int k0 = kc * OZ_KC + kg * 8;
                    const double* col = nullptr;
                    if (E > -100000) {
                        const int u = t.u0 + c / t.nr, r = t.r0 + c % t.nr;
                        col = a.in + (long long)r * a.in_rs + (long long)u * a.in_us + a.in_off + t.off;
                    }
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        neg[e] = false;
                        x[e] = (col != nullptr && k0 + e < K) ? fixed_of(col[k0 + e], E, sb, neg[e]) : 0ULL;
                    }
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        unsigned short h[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            h[e] = bf16_of_digit((unsigned)(x[e] >> ((S - 1 - s) * beta)) & mask, neg[e]);
                        uint4 v;
                        v.x = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
                        v.y = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
                        v.z = (uint32_t)h[4] | ((uint32_t)h[5] << 16);
                        v.w = (uint32_t)h[6] | ((uint32_t)h[7] << 16);
                        *reinterpret_cast<uint4*>(Bd + (long long)s * N * OZ_KC + blk_off(c, kg * 8)) = v;
                    }
                }
                proxy_fence();
                tc_fence_before();
                __syncthreads();
                tc_fence_after();
            }
            if (tid == 0) {
                // digit s of A is in buffer s & 1; digit s + 1 is loaded into the
                // other buffer once the products of digit s - 1 (which read it)
                // have completed, while those of digit s keep the tensor pipe busy
                const unsigned short* Ablk = Am + (long long)((mt * kcn + kc) * S) * OZ_BLOCK;
                mbar_expect_tx(&full[0], OZ_BLOCK * 2);
                bulk_load(Ad, Ablk, OZ_BLOCK * 2, &full[0]);
                for (int s = 0; s < S; ++s) {
                    const int b = s & 1;
                    if (!mbar_wait(&full[b], ph_full[b])) { atomicCAS(z.err, 0, 2); fail = 1; break; }
                    ph_full[b] ^= 1u;
                    tc_fence_after();
                    // descriptors advance by 256 B (two core matrices) per K-step:
                    // +16 in the start-address field
                    const uint64_t ad0 = mat_desc(smem_addr(Ad + b * OZ_BLOCK), 128, 2048);
                    for (int tt = 0; tt + s < S; ++tt) {
                        const uint64_t bd0 = bdesc0 + (uint64_t)((tt * N * OZ_KC * 2) >> 4);
                        const uint32_t dcol = tbase + (uint32_t)((s + tt) * N);
#pragma unroll
                        for (int ks = 0; ks < OZ_KC / 16; ++ks) {
                            const uint32_t acc = (kc > 0 || s > 0 || ks > 0) ? 1u : 0u;
                            mma_bf16(dcol, ad0 + (uint64_t)(ks * 16), bd0 + (uint64_t)(ks * 16), idesc, acc);
                        }
                    }
                    mma_commit(&done[b]);
                    if (s + 1 < S) {
                        if (s >= 1) {
                            if (!mbar_wait(&done[b ^ 1], ph_done[b ^ 1])) { atomicCAS(z.err, 0, 2); fail = 1; break; }
                            ph_done[b ^ 1] ^= 1u;
                        }
                        mbar_expect_tx(&full[b ^ 1], OZ_BLOCK * 2);
                        bulk_load(Ad + (b ^ 1) * OZ_BLOCK, Ablk + (long long)(s + 1) * OZ_BLOCK, OZ_BLOCK * 2, &full[b ^ 1]);
                    }
                }
                if (!fail) mma_commit(chunk);
            }
            __syncthreads();
            if (fail) break;
            // every MMA issued so far is complete once the chunk barrier flips
            if (!mbar_wait(chunk, ph_chunk)) {
                atomicCAS(z.err, 0, 2);
                fail = 1;
            }
            ph_chunk ^= 1u;
            if (tid == 0) {   // the buffer commits of the last two digits completed with the chunk
                for (int s = (S >= 2 ? S - 2 : 0); s < S; ++s) ph_done[s & 1] ^= 1u;
            }
            tc_fence_after();
            __syncthreads();
        }
        if (fail) break;
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (row
        // mt * 128 + 32 (w % 4) + lane) for the columns of its half of the tile,
        // 16 at a time, S diagonals each, and combines them in 64-bit integers
        const int row = mt * 128 + 32 * (warp & 3) + lane;
        const int lo_r = a.row_lo[t.mat], hi_r = a.row_hi[t.mat];
        const bool live_row = row < M && row >= lo_r && row < hi_r;
        const int Ea = z.rexp[(long long)t.mat * z.rexp_stride + row];
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const int half = N / 2, c_lo = (warp >> 2) * half;
        for (int cb = c_lo; cb < c_lo + half; cb += 16) {
            long long hi[16], lo[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) { hi[i] = 0; lo[i] = 0; }
#pragma unroll
            for (int d = 0; d < S; ++d) {
                float f[16];
                tmem_ld16(tbase + lane_base + (uint32_t)(d * N + cb), f);
                if (d < dm) {
                    const int sh = (dm - 1 - d) * beta;
#pragma unroll
                    for (int i = 0; i < 16; ++i) hi[i] += (long long)__float2int_rn(f[i]) << sh;
                } else {
                    const int sh = (S - 1 - d) * beta;
#pragma unroll
                    for (int i = 0; i < 16; ++i) lo[i] += (long long)__float2int_rn(f[i]) << sh;
                }
            }
            if (!live_row) continue;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = cb + i;
                if (c >= ncol || colE[c] <= -100000) continue;
                const int u = t.u0 + c / t.nr, r = t.r0 + c % t.nr;
                // y = 2^e0 (hi 2^((S - dm) beta) + lo): exact conversions of the
                // integers, scaled by exact powers of two (one rounding, in the FMA)
                const int el = Ea + colE[c] - (S + 1) * beta, eh = el + (S - dm) * beta;
                double y;
                if (el >= -1022 && eh <= 1023) {
                    const double ph = __longlong_as_double((long long)(eh + 1023) << 52);
                    const double pl = __longlong_as_double((long long)(el + 1023) << 52);
                    y = fma((double)hi[i], ph, (double)lo[i] * pl);
                } else {
                    y = ldexp((double)hi[i], eh) + ldexp((double)lo[i], el);
                }
                const long long base = (long long)r * a.out_rs + (long long)u * a.out_us + t.off;
                const long long addr = base + (row < a.msplit ? a.out_off0 + row : a.out_off1 + (row - a.msplit));
                if (z.epi == 1) y += a.add[addr];
                a.out[addr] = y;
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    tc_fence_before();
    __syncthreads();
    if (fail && tid == 0)   // bounded grace period for tensor-core work still in flight
        for (int i = 0; i < 1000; ++i) __nanosleep(1000);
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tbase), "r"(512) : "memory");
}

int oz_smem_bytes(int S, int N) { return OzSmemLayout(S, N).total; }

void k_oz_split_rows(const double* mats, long long mat_stride, int nmat, int M, int K, int S, int beta, int mt_n,
                     int kcn, unsigned short* dig, long long dig_stride, int* rexp, long long rexp_stride,
                     cudaStream_t s) {
    const long long warps = (long long)nmat * mt_n * 128;
    oz_split_rows_kernel<double><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(
        mats, mat_stride, nmat, M, K, S, beta, mt_n, kcn, dig, dig_stride, rexp, rexp_stride);
    count_launches(1);
}

void k_oz_split_rows_f(const float* mats, long long mat_stride, int nmat, int M, int K, int S, int beta, int mt_n,
                       int kcn, unsigned short* dig, long long dig_stride, int* rexp, long long rexp_stride,
                       cudaStream_t s) {
    const long long warps = (long long)nmat * mt_n * 128;
    oz_split_rows_kernel<float><<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(
        mats, mat_stride, nmat, M, K, S, beta, mt_n, kcn, dig, dig_stride, rexp, rexp_stride);
    count_launches(1);
}

template <int S, int BETA, int N>
static bool launch_oz_t(const OzArgs& z, const Tile* d_tiles, int ntiles, cudaStream_t s) {
    const int smem = oz_smem_bytes(S, N);
    static int configured = 0;
    if (configured < smem) {
        if (cudaFuncSetAttribute(oz_gemm_kernel<S, BETA, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
            return false;
        configured = smem;
    }
    oz_gemm_kernel<S, BETA, N><<<ntiles, OZ_THREADS, smem, s>>>(z, d_tiles);
    count_launches(1);
    return cudaPeekAtLastError() == cudaSuccess;
}

bool launch_oz_gemm(const OzArgs& z, const Tile* d_tiles, int ntiles, cudaStream_t s) {
    if (ntiles <= 0) return true;
    if (z.S == 8 && z.beta == 7 && z.N == 64) return launch_oz_t<8, 7, 64>(z, d_tiles, ntiles, s);
    if (z.S == 10 && z.beta == 6 && z.N == 32) return launch_oz_t<10, 6, 32>(z, d_tiles, ntiles, s);
    if (z.S == 12 && z.beta == 5 && z.N == 32) return launch_oz_t<12, 5, 32>(z, d_tiles, ntiles, s);
    if (z.S == 4 && z.beta == 7 && z.N == 64) return launch_oz_t<4, 7, 64>(z, d_tiles, ntiles, s);
    if (z.S == 4 && z.beta == 6 && z.N == 64) return launch_oz_t<4, 6, 64>(z, d_tiles, ntiles, s);
    if (z.S == 5 && z.beta == 5 && z.N == 64) return launch_oz_t<5, 5, 64>(z, d_tiles, ntiles, s);
    return false;
}

// Digit-size choice for K: the largest beta <= 7 with S = ceil(bits / beta)
// digits such that S K (2^beta - 1)^2 < 2^24 (exact FP32 accumulation of a
// whole anti-diagonal over all of K); N = 64 columns per tile for S <= 8,
// 32 above (S N <= 512 tensor-memory columns).  bits = 56 gives FP64
// accuracy, bits = 24 the 24-bit significand of FP32 (the products that
// replace FP32 CUDA-core products).
bool oz_choose(int K, int& S, int& beta, int& N, int bits) {
    for (beta = 7; beta >= 5; --beta) {
        S = (bits + beta - 1) / beta;
        const double bound = (double)S * K * (double)((1 << beta) - 1) * (double)((1 << beta) - 1);
        if (bound < 16777216.0) {
            N = S <= 8 ? 64 : 32;
            return S * N <= 512;
        }
    }
    return false;
}

}  // namespace smpm

// Tensor-core contraction engine for sm_103a (tcgen05 + TMEM + TMA).
//
// C[m][n] = alpha * sum_k A[m][k] B[n][k] + beta * C with A, B in BF16,
// K-major, staged in shared memory by TMA (128-byte swizzle) through a
// 4-stage mbarrier pipeline and multiplied by tcgen05.mma (kind::f16,
// M = 128, N = 128/256, K = 16 per instruction) into an FP32 accumulator in
// tensor memory.  Warp roles: warp 0 issues TMA loads, warp 1 owns TMEM and
// issues the MMAs (one thread), warps 2-5 drain TMEM with tcgen05.ld and
// write the tile (FP64 C through arbitrary strides, or BF16 directly in the
// packed operand layout of a following GEMM).
//
// Precision: operands are rounded to BF16 (nsplit = 1) or split x = hi + lo
// with hi, lo BF16 (nsplit = 2) and multiplied as hi*hi + hi*lo + lo*hi by
// concatenating three segments along K (A: [hi|hi|lo], B: [hi|lo|hi]); the
// accumulation is FP32 in TMEM, the result is added to the FP64 residual.
//
// Every mbarrier wait is bounded (about two seconds of wall time); on
// expiry the kernel records an error flag, waits (bounded) for its own
// copies and MMAs in flight, frees its TMEM and returns.
#include "common.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

namespace dcsd {

// ---------------------------------------------------------------------------
// device helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 0 && gtimer() - t0 > kWaitNs) return false;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}
// K-blocked operand [k block][row][64]: coordinates (0, row, k block)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
// the same load delivered to the same shared-memory offset of every CTA in
// ctaMask (this GPU's own memory; cluster of two CTAs), completing bytes on
// the mbarrier at the same offset in each
__device__ __forceinline__ void tma_load_3d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                               uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.multicast::cluster"
        " [%0], [%1, {%3, %4, %5}], [%2], %6;" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z), "h"(mask)
        : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// completion of the issued MMAs signalled on the mbarrier at the same offset
// in every CTA of ctaMask
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// K-major operand tile: rows of 64 BF16 (128 B), 128-byte swizzle, 8-row
// atoms of 1024 B (stride-dimension byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= 1ull << 46;
    d |= 2ull << 61;
    return d;
}

constexpr int TC_BM = 128, TC_BK = 64, TC_STAGES = 4;

// x = hi + mid + lo with each part BF16 (8 significant bits each)
__device__ __forceinline__ __nv_bfloat16 split_part(float x, int part) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    if (part == 0) return hi;
    const float r1 = x - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    if (part == 1) return mid;
    return __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

struct TcEpi {
    int mode;               // 0: FP64 C (alpha, beta); 4: FP32 C32 += alpha * acc;
                            // 5: split-K FP32 partial tiles into C32;
                            // 1: BF16 packed output;
                            // 2: ladder producer tile, staged through shared memory
                            //    and stored as 16-byte vectors (see ladder_tc)
    double* C;
    float* C32;             // mode 4 output; mode 3: FP32 scatter target when set
    __nv_bfloat16* P;
    double alpha, beta;
    int nm, nn;
    long m_size[kMaxMode], m_s[kMaxMode];
    long n_size[kMaxMode], n_s[kMaxMode];
    long M, N;
    int nseg;               // modes 1/2: segments written (1, 3 or 6)
    long segstride;         // modes 1/2: elements between segments
    int pat[6];             // modes 1/2: part per segment, 0 = hi, 1 = mid, 2 = lo
    // mode 2: row m = (r, c) with c < V; column n = (b', d) with d < Vp;
    //         element -> P[(r*Vb + b')*rowlen + c*Vp + d]
    long V, Vp, rowlen, Vb;
    // mode 2 with kbs > 0: K-blocked destination, element (row R, k) at
    //         P[(k / 64) * kbs + R * 64 + k % 64] (+ segment * segstride)
    long kbs;
    // mode 3: ladder consumer scatter; row m = (s, i, j), column n = (r, b')
    //         with a = a0 + r, b = a0 + b' (only b >= a is used):
    //         s = 0,1 (same spin): R[s][ij][a][b] += v, R[s][ij][b][a] -= v
    //         s = 2 (ab):           R[2][ij][a][b] += v
    //         s = 3 (ab, (c,d) exchanged): R[2][ij][b][a] += v  (b > a)
    //         s = 4, 5 (ab, S+ and S- of the symmetric / antisymmetric form)
    // mode 6: G-pass scatter of the symmetric / antisymmetric form (C = G)
    long a0, OO, VV;
    long O;
    const int* rowcode;     // mode 3: row -> (block << 20 | i << 10 | j); same-spin rows are pairs i < j
    const long* mrow;       // modes 0/4: row -> offset in C (replaces the m-mode decomposition)
};

// ladder consumer scatter of one accumulator element v = W(a,b) for the row
// (blk, i, j); same-spin blocks hold the pair i < j only and also fill the
// (j, i) row: R[ij][ab] = -R[ij][ba] = -R[ji][ab] = R[ji][ba]
// Rows of the symmetric / antisymmetric form (blocks 4 and 5, alpha-beta):
// S+ adds to R[ij][ab] and R[ij][ba], S- adds to R[ij][ab] and subtracts
// from R[ij][ba] (S- vanishes at a = b).
// Every target of a launch receives one update (the targets of different
// rows and columns are distinct; a = b same-spin elements are skipped, their
// four updates cancel), so the updates are reductions without a returned
// value: the result equals a read-modify-write and no load is waited for.
template <typename T>
__device__ __forceinline__ void ladder_scatter(T* R, int sblk, long ro1, long ro2, long a, long b, long V, T v) {
    if (b < a) return;
    if (sblk < 2) {
        if (b == a) return;
        atomicAdd(R + ro1 + a * V + b, v);
        atomicAdd(R + ro1 + b * V + a, -v);
        atomicAdd(R + ro2 + a * V + b, -v);
        atomicAdd(R + ro2 + b * V + a, v);
    } else if (sblk == 2) {
        atomicAdd(R + ro1 + a * V + b, v);
    } else if (sblk == 4) {
        atomicAdd(R + ro1 + a * V + b, v);
        if (b > a) atomicAdd(R + ro1 + b * V + a, v);
    } else if (sblk == 5) {
        if (b > a) {
            atomicAdd(R + ro1 + a * V + b, v);
            atomicAdd(R + ro1 + b * V + a, -v);
        }
    } else if (b > a) {
        atomicAdd(R + ro1 + b * V + a, v);
    }
}

__device__ __forceinline__ long decomp1(long idx, int nmode, const long* size, const long* s) {
    long o = 0;
#pragma unroll
    for (int j = kMaxMode - 1; j >= 0; --j) {
        if (j < nmode) {
            long q = idx / size[j];
            o += (idx - q * size[j]) * s[j];
            idx = q;
        }
    }
    return o;
}

// offset of a linear index over up to kMaxMode modes (last mode fastest);
// indices and mode sizes are below 2^31, so the divisions are 32-bit
__device__ __forceinline__ long decomp1_u32(unsigned idx, int nmode, const long* size, const long* s) {
    long o = 0;
#pragma unroll
    for (int j = kMaxMode - 1; j >= 0; --j) {
        if (j < nmode) {
            const unsigned sz = (unsigned)size[j];
            const unsigned q = idx / sz;
            o += (long)(idx - q * sz) * s[j];
            idx = q;
        }
    }
    return o;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int kEpiWarps = 8;  // two warps per TMEM lane quarter, each on half of the columns
constexpr int kTcThreads = 32 * (2 + kEpiWarps);
constexpr int kStageBytesMode2 = kEpiWarps * 32 * 64 * 2;  // epilogue staging, per warp 2 halves x 32 rows x 64 B

// Persistent tcgen05 GEMM: one CTA per SM walks the output tiles (m fastest);
// Output tile of a linear (m, n) tile index in grouped order: bands of
// `group` m-tiles, n-tiles running within a band, so that the CTAs of one
// wave share a compact block of A rows and B rows in L2.
__device__ __forceinline__ void tile_mn(int mn, int tilesM, int tilesN, int group, int& tm, int& tn) {
    const int g = max(1, min(group, tilesM));
    const int band = mn / (g * tilesN), r = mn - band * g * tilesN;
    const int rows = min(g, tilesM - band * g);
    tm = band * g + r % rows;
    tn = r / rows;
}

// two TMEM accumulators of BN columns let the epilogue of one tile overlap
// the MMAs of the next.
//
// MC: launched in clusters of two CTAs that take the two m-tiles of a pair
// with the same n-tile.  Each CTA loads its own A tile and half of the B tile
// (BN / 2 rows; tmB's box is that half) and multicasts the half to both, so
// the pair fetches each B tile from L2 once.  A stage slot is free only when
// both CTAs' MMAs have consumed it: the MMA completion is signalled on the
// empty barrier of both CTAs (count 2), and every TMA issue waits for it.
template <int BN, bool MC>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcEpi epi,
              int nkt, int tilesM, int tilesN, int kper, int group, int kblk, int* err) {
    constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2, B_BYTES = BN * TC_BK * 2;
    constexpr uint32_t STAGE = A_BYTES + B_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* staging = smem + TC_STAGES * STAGE;
    uint64_t* full = (uint64_t*)(staging + kStageBytesMode2);
    uint64_t* empty = full + TC_STAGES;
    uint64_t* accf = empty + TC_STAGES;  // [2] MMA -> epilogue
    uint64_t* acce = accf + 2;           // [2] epilogue -> MMA
    uint32_t* tslot = (uint32_t*)(acce + 2);
    volatile int* issued = (volatile int*)(tslot + 1);
    volatile int* consumed = issued + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tiles enumerate (m tile, n tile, k split); split s covers the k-steps
    // [s * kper, min(nkt, (s + 1) * kper)).  MC: the schedule runs over pairs
    // of m-tiles (the pair's CTA of rank r takes m-tile 2 * pair + r; an
    // m-tile beyond the last one reads zeros and stores nothing)
    const int crank = MC ? (int)cluster_rank() : 0;
    const int tile0 = MC ? (int)blockIdx.x / 2 : (int)blockIdx.x;
    const int tstep = MC ? (int)gridDim.x / 2 : (int)gridDim.x;
    const int tilesMs = MC ? (tilesM + 1) / 2 : tilesM;
    const int nmn = tilesMs * tilesN;
    const int ntiles = nmn * ((nkt + kper - 1) / kper);
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], MC ? 2 : 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kEpiWarps);
        }
        *issued = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tslot, 2 * BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // MC: the peer's barriers are initialised before any multicast reaches them
    if (MC) cluster_sync();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int tile = tile0; tile < ntiles && ok; tile += tstep) {
                const int mn = tile % nmn, ks = tile / nmn;
                int tm, tn;
                tile_mn(mn, tilesMs, tilesN, group, tm, tn);
                if (MC) tm = 2 * tm + crank;
                const int m0 = tm * TC_BM, n0 = tn * BN;
                const int kb = ks * kper, ke = min(nkt, kb + kper);
                for (int kt = kb; kt < ke; ++kt, ++g) {
                    const int s = g % TC_STAGES, round = g / TC_STAGES;
                    if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1)) {
                        atomicExch(err, 1);
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], STAGE);
                    if (MC) {
                        tma_load_3d(smem + s * STAGE, &tmA, &full[s], 0, m0, kt);
                        tma_load_3d_mc(smem + s * STAGE + A_BYTES + crank * (B_BYTES / 2), &tmB, &full[s], 0,
                                       n0 + crank * (BN / 2), kt, (uint16_t)0x3);
                    } else if (kblk) {
                        tma_load_3d(smem + s * STAGE, &tmA, &full[s], 0, m0, kt);
                        tma_load_3d(smem + s * STAGE + A_BYTES, &tmB, &full[s], 0, n0, kt);
                    } else {
                        tma_load_2d(smem + s * STAGE, &tmA, &full[s], kt * TC_BK, m0);
                        tma_load_2d(smem + s * STAGE + A_BYTES, &tmB, &full[s], kt * TC_BK, n0);
                    }
                    *issued = g + 1;
                }
            }
            if (MC) {
                // every slot free in both CTAs: the peer's last MMA completions
                // have arrived here and no multicast of this CTA is pending
                const int g0 = max(0, g - TC_STAGES);
                for (int gg = g0; gg < g; ++gg)
                    if (!mbar_wait(&empty[gg % TC_STAGES], (gg / TC_STAGES) & 1)) atomicExch(err, 5);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                       ((uint32_t)(TC_BM >> 4) << 24);
            int g = 0, j = 0;
            bool ok = true;
            for (int tile = tile0; tile < ntiles && ok; tile += tstep, ++j) {
                const int buf = j & 1, u = j >> 1;
                if (u > 0 && !mbar_wait(&acce[buf], (u - 1) & 1)) {
                    atomicExch(err, 4);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * BN);
                const int kb = (tile / nmn) * kper, ke = min(nkt, kb + kper);
                for (int kt = kb; kt < ke; ++kt, ++g) {
                    const int s = g % TC_STAGES, round = g / TC_STAGES;
                    if (!mbar_wait(&full[s], round & 1)) {
                        atomicExch(err, 2);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk)
                        mma_bf16(d, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), idesc,
                                 (kt > kb || kk > 0) ? 1u : 0u);
                    if (MC) mma_commit_mc(&empty[s], (uint16_t)0x3);
                    else mma_commit(&empty[s]);
                    *consumed = g + 1;
                }
                if (ok) mma_commit(&accf[buf]);
            }
            if (!ok) {
                // let issued MMAs finish and drain copies that were not consumed
                uint64_t* fin = &accf[j & 1];
                mma_commit(fin);
                for (int kt = *consumed; kt < *issued; ++kt) mbar_wait(&full[kt % TC_STAGES], (kt / TC_STAGES) & 1);
            }
        }
    } else {
        // epilogue warps 2..9 -> TMEM lane quarter (warp % 4); warps 2..5 take
        // the first half of the tile's columns, warps 6..9 the second
        const int q = warp & 3;
        const int ch0 = ((warp - 2) >> 2) * (BN / 64), ch1 = ch0 + BN / 64;
        int j = 0;
        for (int tile = tile0; tile < ntiles; tile += tstep, ++j) {
            const int buf = j & 1, u = j >> 1;
            const int mn = tile % nmn, ksp = tile / nmn;
            int tm, tn;
            tile_mn(mn, tilesMs, tilesN, group, tm, tn);
            if (MC) tm = 2 * tm + crank;
            const int m0 = tm * TC_BM, n0 = tn * BN;
            const bool ok = mbar_wait(&accf[buf], u & 1);
            tc_fence_after();
            if (!ok) {
                atomicExch(err, 3);
                break;
            }
            const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * BN);
            if (epi.mode == 5) {
                // split-K partial: ws[(split * N + n) * M + m], lanes along m
                const long m = (long)m0 + 32 * q + lane;
                float* ws = epi.C32 + (long)ksp * epi.N * epi.M + m;
#pragma unroll 1
                for (int ch = ch0; ch < ch1; ++ch) {
                    uint32_t r[32];
                    tmem_ld32(tbase + (uint32_t)(ch * 32), r);
                    if (m >= epi.M) continue;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        const long nn = (long)n0 + ch * 32 + jj;
                        if (nn < epi.N) ws[nn * epi.M] = __uint_as_float(r[jj]);
                    }
                }
            } else if (epi.mode == 2) {
                // lane = row; BF16 conversion staged through shared memory, then
                // each row's 64 contiguous bytes go out as four 16-byte vectors,
                // 8 rows per warp instruction
                uint4* stage = (uint4*)(staging + (warp - 2) * 32 * 64 * 2);
                const long m = (long)m0 + 32 * q + lane;
                const long r_of = m / epi.V, c_of = m - r_of * epi.V;
                const long rowR = r_of * epi.Vb, colK = c_of * epi.Vp;  // destination row / k of b' = d = 0
                const float alpha = (float)epi.alpha;
#pragma unroll 1
                for (int ch = ch0; ch < ch1; ++ch) {
                    uint32_t rr[32];
                    tmem_ld32(tbase + (uint32_t)(ch * 32), rr);
                    const long nst = (long)n0 + ch * 32;
                    for (int sgm = 0; sgm < epi.nseg; ++sgm) {
                        uint32_t w[16];
#pragma unroll
                        for (int jj = 0; jj < 32; jj += 2) {
                            uint32_t two[2];
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                const float x = alpha * __uint_as_float(rr[jj + t]);
                                two[t] = (uint32_t)__bfloat16_as_ushort(split_part(x, epi.pat[sgm]));
                            }
                            w[jj / 2] = two[0] | (two[1] << 16);
                        }
                        uint4* row = stage + (sgm & 1) * 128 + lane * 4;
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            row[v] = make_uint4(w[4 * v], w[4 * v + 1], w[4 * v + 2], w[4 * v + 3]);
                        __syncwarp();
#pragma unroll
                        for (int it = 0; it < 4; ++it) {
                            const int rrow = it * 8 + (lane >> 2), piece = lane & 3;
                            const long bR = __shfl_sync(0xffffffffu, rowR, rrow);
                            const long bK = __shfl_sync(0xffffffffu, colK, rrow);
                            const long mrow = (long)m0 + 32 * q + rrow;
                            const long np = nst + piece * 8;
                            if (mrow < epi.M && np < epi.N) {
                                const long b = np / epi.Vp, dd = np - b * epi.Vp;
                                const long R = bR + b, k = bK + dd;  // k is a multiple of 8
                                const long off = epi.kbs > 0 ? (k >> 6) * epi.kbs + R * 64 + (k & 63)
                                                             : R * epi.rowlen + k;
                                const uint4 val = stage[(sgm & 1) * 128 + rrow * 4 + piece];
                                *(uint4*)(epi.P + off + sgm * epi.segstride) = val;
                            }
                        }
                        __syncwarp();
                    }
                }
            } else if (epi.mode == 3) {
                const long m = (long)m0 + 32 * q + lane;
                const bool rowok = m < epi.M;
                const int code = rowok ? epi.rowcode[m] : 0;
                const int sblk = code >> 20, ri = (code >> 10) & 1023, rj = code & 1023;
                const long blkoff = (long)(sblk < 2 ? sblk : 2) * epi.OO * epi.VV;
                const long ro1 = blkoff + ((long)ri * epi.O + rj) * epi.VV;
                const long ro2 = blkoff + ((long)rj * epi.O + ri) * epi.VV;
#pragma unroll 1
                for (int ch = ch0; ch < ch1; ++ch) {
                    uint32_t r[32];
                    tmem_ld32(tbase + (uint32_t)(ch * 32), r);
                    if (!rowok) continue;
                    const long nst = (long)n0 + ch * 32;
                    long rr = nst / epi.Vb, bb = nst - rr * epi.Vb;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        if (nst + jj < epi.N) {
                            const long a = epi.a0 + rr, b = epi.a0 + bb;
                            if (epi.C32)
                                ladder_scatter<float>(epi.C32, sblk, ro1, ro2, a, b, epi.V, __uint_as_float(r[jj]));
                            else
                                ladder_scatter<double>(epi.C, sblk, ro1, ro2, a, b, epi.V,
                                                       (double)__uint_as_float(r[jj]));
                        }
                        if (++bb == epi.Vb) { bb = 0; ++rr; }
                    }
                }
            } else if (epi.mode == 6) {
                // G-pass scatter of the symmetric / antisymmetric form: row m =
                // (blk, i, j) as in mode 3, column n = (r, b) with k = a0 + r;
                // G[s][i][j][k][b] at ((s O + i) O + j) O V + k V + b.  Blocks
                // 0/1 add to their own G block, 4 (S+) adds to G[2] and G[3],
                // 5 (S-) adds to G[2] and subtracts from G[3]
                const long m = (long)m0 + 32 * q + lane;
                const bool rowok = m < epi.M;
                const int code = rowok ? epi.rowcode[m] : 0;
                const int sblk = code >> 20, ri = (code >> 10) & 1023, rj = code & 1023;
                const long OV = epi.O * epi.V;
                const long g1 = (((long)(sblk < 2 ? sblk : 2) * epi.O + ri) * epi.O + rj) * OV;
                const long g3 = ((3l * epi.O + ri) * epi.O + rj) * OV;
#pragma unroll 1
                for (int ch = ch0; ch < ch1; ++ch) {
                    uint32_t r[32];
                    tmem_ld32(tbase + (uint32_t)(ch * 32), r);
                    if (!rowok) continue;
                    const long nst = (long)n0 + ch * 32;
                    long rr = nst / epi.Vb, bb = nst - rr * epi.Vb;
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        if (nst + jj < epi.N) {
                            const long off = (epi.a0 + rr) * epi.V + bb;
                            // one update per target and launch: reductions
                            const double v = (double)__uint_as_float(r[jj]);
                            atomicAdd(epi.C + g1 + off, v);
                            if (sblk == 4) atomicAdd(epi.C + g3 + off, v);
                            else if (sblk == 5) atomicAdd(epi.C + g3 + off, -v);
                        }
                        if (++bb == epi.Vb) { bb = 0; ++rr; }
                    }
                }
            } else {
                const long m = (long)m0 + 32 * q + lane;
                const bool rowok = m < epi.M;
                const long roff = !rowok ? 0 : epi.mrow ? epi.mrow[m] : decomp1(m, epi.nm, epi.m_size, epi.m_s);
                const float alpha = (float)epi.alpha;
                // offsets in C of this warp's columns, once per tile, kept in
                // the warp's staging slot (-1: column outside C)
                long* coffs = (long*)(staging + (warp - 2) * 32 * 64 * 2);
                for (int cc = lane; cc < (ch1 - ch0) * 32; cc += 32) {
                    const long nidx = (long)n0 + ch0 * 32 + cc;
                    coffs[cc] = nidx < epi.N ? decomp1_u32((unsigned)nidx, epi.nn, epi.n_size, epi.n_s) : -1;
                }
                __syncwarp();
#pragma unroll 1
                for (int ch = ch0; ch < ch1; ++ch) {
                    uint32_t r[32];
                    tmem_ld32(tbase + (uint32_t)(ch * 32), r);
                    if (!rowok) continue;
                    const long* cb = coffs + (ch - ch0) * 32;
                    if (epi.mode == 0 && epi.beta == 1.0) {
                        // FP64 accumulation with beta = 1: one update per element
                        // and launch, as a reduction (old + v, as fma(1, old, v))
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            const long co = cb[jj];
                            if (co >= 0) atomicAdd(epi.C + roff + co, f32_to_f64(alpha * __uint_as_float(r[jj])));
                        }
                        continue;
                    }
                    if (epi.mode == 4) {
                        // FP32 accumulation: every element of C32 gets one update
                        // per launch, as a reduction (no load waited for)
#pragma unroll
                        for (int jj = 0; jj < 32; ++jj) {
                            const long co = cb[jj];
                            if (co >= 0) atomicAdd(epi.C32 + roff + co, alpha * __uint_as_float(r[jj]));
                        }
                        continue;
                    }
                    // two halves of 16 columns: all loads of a half, then its stores
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        if (epi.mode == 4) {
                            float oldf[16];
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const long co = cb[h * 16 + jj];
                                oldf[jj] = co >= 0 ? epi.C32[roff + co] : 0.0f;
                            }
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const long co = cb[h * 16 + jj];
                                if (co >= 0) epi.C32[roff + co] = fmaf(alpha, __uint_as_float(r[h * 16 + jj]), oldf[jj]);
                            }
                        } else if (epi.mode == 0) {
                            double old[16];
                            if (epi.beta != 0.0) {
#pragma unroll
                                for (int jj = 0; jj < 16; ++jj) {
                                    const long co = cb[h * 16 + jj];
                                    old[jj] = co >= 0 ? epi.C[roff + co] : 0.0;
                                }
                            }
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const long co = cb[h * 16 + jj];
                                if (co < 0) continue;
                                const double v = f32_to_f64(alpha * __uint_as_float(r[h * 16 + jj]));
                                epi.C[roff + co] = epi.beta != 0.0 ? fma(epi.beta, old[jj], v) : v;
                            }
                        } else {
#pragma unroll
                            for (int jj = 0; jj < 16; ++jj) {
                                const long co = cb[h * 16 + jj];
                                if (co < 0) continue;
                                const float v = alpha * __uint_as_float(r[h * 16 + jj]);
                                for (int sgm = 0; sgm < epi.nseg; ++sgm)
                                    epi.P[roff + co + sgm * epi.segstride] = split_part(v, epi.pat[sgm]);
                            }
                        }
                    }
                }
                __syncwarp();  // the next tile rewrites coffs
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    __syncwarp();
    if (MC) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

// ---------------------------------------------------------------------------
// ladder in symmetric / antisymmetric form
// ---------------------------------------------------------------------------
// For a <= b and c <= d: M+_ab[cd] = (ac|bd) + (ad|bc), M-_ab[cd] = (ac|bd) -
// (ad|bc).  With A+[cd] = (t_cd + t_dc) / 2 (t_cc / 2 on the diagonal) and
// A-[cd] = (t_cd - t_dc) / 2, sum_cd t_cd (ac|bd) = S+ + S- and
// sum_cd t_cd (bc|ad) = S+ - S-, S+- = sum_{c<=d} A+- M+-: the contraction runs
// over half of the (c,d) pairs.  The (c <= d) index is compact: row c holds
// d in [floor8(c), Vp), so that 8 consecutive d stay 16-byte aligned;
// entries with d < c meet zero amplitudes.
__host__ __device__ __forceinline__ long sa_koff(long c, long Vp) {
    const long g = c >> 3, rem = c & 7;
    return 8 * (g * Vp - 4 * g * (g - 1)) + rem * (Vp - 8 * g);
}

constexpr int SA_STAGES = 3;
constexpr uint32_t SA_TILE = 128 * TC_BK * 2;  // one 128-row operand tile (16 KB)

struct SaArgs {
    int nkt;              // k-steps over the packed L (segments x L / 64)
    int nr, Vb, nblk;     // chunk rows, columns b, 128-wide c/d blocks
    int npair;            // (C, D) block pairs with C <= D
    long ntiles;          // npair x #(r, b'): b' >= r (ladder) or all (rect)
    int rect;             // 0: the ladder triangle b' >= r; 1: all (r, b') (G pass)
    int xa0, xb0;         // orbital of row r = 0 and of column b' = 0
    int YP;               // packed rows per orbital (multiple of 128)
    int V, Vp;
    long kbs;             // k-block stride of a V tile (vrows * 64)
    long segstride;       // elements between the segments of a V tile
    int nseg, pat[6];
    __nv_bfloat16* Vplus;
    __nv_bfloat16* Vminus;
};

// Tile t -> (r, b', C, D): (C, D) fastest, then r, then b' (b' >= r), so
// that the tiles in flight share the rows of one b and the chunk's few a
// rows stay in L2 (each b's rows are read from memory once per chunk)
__device__ __forceinline__ void sa_tile(const SaArgs& a, long t, int& r, int& bb, int& C, int& D) {
    long u = t / a.npair;
    int pr = (int)(t - u * a.npair);
    const long tri = (long)a.nr * (a.nr + 1) / 2;  // b' < nr: r in [0, b']
    if (a.rect) {
        bb = (int)(u / a.nr);
        r = (int)(u % a.nr);
    } else if (u < tri) {
        bb = 0;
        while (u >= bb + 1) {
            u -= bb + 1;
            ++bb;
        }
        r = (int)u;
    } else {
        u -= tri;
        bb = a.nr + (int)(u / a.nr);
        r = (int)(u % a.nr);
    }
    C = 0;
    while (pr >= a.nblk - C) {
        pr -= a.nblk - C;
        ++C;
    }
    D = C + pr;
}

// Producer of the M+ and M- tiles of one chunk of a: tile (a, b, C, D) with
// b >= a and C <= D, two accumulators acc1 = B_a[C] B_b[D]^T = M_ab[C][D] and
// acc2 = B_b[C] B_a[D]^T (element (c,d) = (ad|bc)).  tmA / tmB: the packed
// virtual-virtual DF factors [(x, y)][L] (y padded to YP rows per x), with
// the A-side and the B-side split patterns, K-blocked.  Pipeline as in
// k_tc_gemm: warp 0 loads four 16 KB tiles per stage, warp 1 issues the
// MMAs, eight epilogue warps write M+- (BF16 split parts) at the compact
// (c <= d) index of V tile row (r, b').
__global__ void __launch_bounds__(kTcThreads, 1)
    k_ladder_sa(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, SaArgs a,
                int* err) {
    constexpr uint32_t STAGE = 4 * SA_TILE;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + SA_STAGES * STAGE);
    uint64_t* empty = full + SA_STAGES;
    uint64_t* accf = empty + SA_STAGES;
    uint64_t* acce = accf + 2;
    uint32_t* tslot = (uint32_t*)(acce + 2);
    volatile int* issued = (volatile int*)(tslot + 1);
    volatile int* consumed = issued + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < SA_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], kEpiWarps);
        }
        *issued = 0;
        *consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tslot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (long t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
                int r, bb, C, D;
                sa_tile(a, t, r, bb, C, D);
                const int xa = (a.xa0 + r) * a.YP, xb = (a.xb0 + bb) * a.YP;
                for (int kt = 0; kt < a.nkt; ++kt, ++g) {
                    const int s = g % SA_STAGES, round = g / SA_STAGES;
                    if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1)) {
                        atomicExch(err, 1);
                        ok = false;
                        break;
                    }
                    // diagonal block (C = D): acc2 = B_b[C] B_a[C]^T uses the same
                    // two tiles as acc1 with the roles swapped
                    uint8_t* st = smem + s * STAGE;
                    if (C == D) {
                        mbar_expect_tx(&full[s], 2 * SA_TILE);
                        tma_load_3d(st, &tmA, &full[s], 0, xa + C * 128, kt);            // B_a[C]
                        tma_load_3d(st + SA_TILE, &tmB, &full[s], 0, xb + D * 128, kt);  // B_b[C]
                    } else {
                        mbar_expect_tx(&full[s], STAGE);
                        tma_load_3d(st, &tmA, &full[s], 0, xa + C * 128, kt);                // B_a[C]
                        tma_load_3d(st + SA_TILE, &tmB, &full[s], 0, xb + D * 128, kt);      // B_b[D]
                        tma_load_3d(st + 2 * SA_TILE, &tmA, &full[s], 0, xb + C * 128, kt);  // B_b[C]
                        tma_load_3d(st + 3 * SA_TILE, &tmB, &full[s], 0, xa + D * 128, kt);  // B_a[D]
                    }
                    *issued = g + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(128 >> 3) << 17) |
                                       ((uint32_t)(TC_BM >> 4) << 24);
            int g = 0, j = 0;
            bool ok = true;
            for (long t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x, ++j) {
                const int buf = j & 1, u = j >> 1;
                if (u > 0 && !mbar_wait(&acce[buf], (u - 1) & 1)) {
                    atomicExch(err, 4);
                    ok = false;
                    break;
                }
                tc_fence_after();
                int r_, bb_, C, D;
                sa_tile(a, t, r_, bb_, C, D);
                // second product's operands: B_b[C], B_a[D] (tiles 2, 3), or
                // for a diagonal block tiles 1 and 0
                const uint32_t o2a = C == D ? SA_TILE : 2 * SA_TILE, o2b = C == D ? 0u : 3 * SA_TILE;
                const uint32_t d1 = tmem + (uint32_t)(buf * 256), d2 = d1 + 128;
                for (int kt = 0; kt < a.nkt; ++kt, ++g) {
                    const int s = g % SA_STAGES, round = g / SA_STAGES;
                    if (!mbar_wait(&full[s], round & 1)) {
                        atomicExch(err, 2);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(smem + s * STAGE);
#pragma unroll
                    for (int kk = 0; kk < TC_BK / 16; ++kk) {
                        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                        mma_bf16(d1, smem_desc(base + kk * 32), smem_desc(base + SA_TILE + kk * 32), idesc, acc);
                        mma_bf16(d2, smem_desc(base + o2a + kk * 32), smem_desc(base + o2b + kk * 32), idesc, acc);
                    }
                    mma_commit(&empty[s]);
                    *consumed = g + 1;
                }
                if (ok) mma_commit(&accf[buf]);
            }
            if (!ok) {
                uint64_t* fin = &accf[j & 1];
                mma_commit(fin);
                for (int kt = *consumed; kt < *issued; ++kt) mbar_wait(&full[kt % SA_STAGES], (kt / SA_STAGES) & 1);
            }
        }
    } else {
        // warps 2..9: TMEM lane quarter warp % 4; warps 2..5 take columns
        // 0..63 of both accumulators, warps 6..9 columns 64..127
        const int q = warp & 3, h = (warp - 2) >> 2;
        int j = 0;
        for (long t = blockIdx.x; t < a.ntiles; t += gridDim.x, ++j) {
            const int buf = j & 1, u = j >> 1;
            int r, bb, C, D;
            sa_tile(a, t, r, bb, C, D);
            const bool ok = mbar_wait(&accf[buf], u & 1);
            tc_fence_after();
            if (!ok) {
                atomicExch(err, 3);
                break;
            }
            const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * 256);
            const long c = (long)C * 128 + 32 * q + lane;
            const long c8 = c & ~7l, kc = sa_koff(c, a.Vp);
            const long R = (long)r * a.Vb + bb;  // V tile row
#pragma unroll 1
            for (int ch = 2 * h; ch < 2 * h + 2; ++ch) {
                uint32_t r1[32], r2[32];
                tmem_ld32(tb + (uint32_t)(ch * 32), r1);
                tmem_ld32(tb + 128u + (uint32_t)(ch * 32), r2);
                if (c >= a.V) continue;
#pragma unroll
                for (int g8 = 0; g8 < 4; ++g8) {
                    const long d = (long)D * 128 + ch * 32 + g8 * 8;
                    if (d < c8 || d >= a.Vp) continue;
                    const long k = kc + (d - c8);
                    const long off = (k >> 6) * a.kbs + R * 64 + (k & 63);
                    float pl[8], mi[8];
#pragma unroll
                    for (int x = 0; x < 8; ++x) {
                        const float v1 = __uint_as_float(r1[g8 * 8 + x]), v2 = __uint_as_float(r2[g8 * 8 + x]);
                        pl[x] = v1 + v2;
                        mi[x] = v1 - v2;
                    }
                    for (int sg = 0; sg < a.nseg; ++sg) {
                        uint32_t wp[4], wm[4];
#pragma unroll
                        for (int x = 0; x < 4; ++x) {
                            wp[x] = (uint32_t)__bfloat16_as_ushort(split_part(pl[2 * x], a.pat[sg])) |
                                    ((uint32_t)__bfloat16_as_ushort(split_part(pl[2 * x + 1], a.pat[sg])) << 16);
                            wm[x] = (uint32_t)__bfloat16_as_ushort(split_part(mi[2 * x], a.pat[sg])) |
                                    ((uint32_t)__bfloat16_as_ushort(split_part(mi[2 * x + 1], a.pat[sg])) << 16);
                        }
                        *(uint4*)(a.Vplus + off + sg * a.segstride) = make_uint4(wp[0], wp[1], wp[2], wp[3]);
                        *(uint4*)(a.Vminus + off + sg * a.segstride) = make_uint4(wm[0], wm[1], wm[2], wm[3]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// Stacked S/A amplitudes from t2 (FP64): operand Am rows [same-spin pairs
// i < j of blocks 0 and 1 (2P); alpha-beta (O^2)] with A-, operand Ap rows
// [alpha-beta (O^2)] with A+, over the compact (c <= d) index, K-blocked
// [Kp / 64][rows][64], nseg segments (pattern pat) `seg*` elements apart.
// Work item: a source row and a 32 x 32 tile of (c, d) with the d tile not
// below the c tile; both orientations of the tile pass through shared memory.
struct SaPackArgs {
    const double* t2;
    const long* pairoff;   // [2P] offsets of the same-spin pair rows
    long OO, VV;
    int P2, V, Vp, ntile;  // 2P, V, Vp, 32-wide tiles over V
    long Kp;
    __nv_bfloat16* Am;
    __nv_bfloat16* Ap;
    long rowsM, rowsP;     // rows of Am (2P + O^2) and Ap (O^2)
    int nseg, pat[6];
};

__global__ void __launch_bounds__(256) k_pack_sa(SaPackArgs a) {
    __shared__ float tcd[32][33], tdc[32][33];
    const long ntp = (long)a.ntile * (a.ntile + 1) / 2;
    const long nsrc = a.P2 + a.OO;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (long w = blockIdx.x; w < nsrc * ntp; w += gridDim.x) {
        const long src = w / ntp;
        long tp = w - src * ntp;
        int tc = 0;
        while (tp >= a.ntile - tc) {
            tp -= a.ntile - tc;
            ++tc;
        }
        const int td = tc + (int)tp;
        const bool ss = src < a.P2;
        const double* T = a.t2 + (ss ? a.pairoff[src] : 2 * a.OO * a.VV + (src - a.P2) * a.VV);
        const int c0 = 32 * tc, d0 = 32 * td;
        // all eight loads of a thread in flight before the first store
        double vcd[4], vdc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int rr = ty + 8 * q;
            const int c = c0 + rr, d = d0 + tx;
            vcd[q] = (c < a.V && d < a.V) ? T[(long)c * a.V + d] : 0.0;      // t[c0+rr][d0+tx]
            const int dd = d0 + rr, cc = c0 + tx;
            vdc[q] = (dd < a.V && cc < a.V) ? T[(long)dd * a.V + cc] : 0.0;  // t[d0+rr][c0+tx]
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            tcd[ty + 8 * q][tx] = f64_to_f32(vcd[q]);
            tdc[ty + 8 * q][tx] = f64_to_f32(vdc[q]);
        }
        __syncthreads();
        // threads 0..127: row c = c0 + tid / 4, 8 d from d0 + 8 * (tid % 4)
        if (threadIdx.x < 128) {
            const int rr = threadIdx.x >> 2, g = threadIdx.x & 3;
            const long c = c0 + rr, c8 = c & ~7l, d = d0 + 8 * g;
            if (c < a.V && d >= c8 && d < a.Vp) {
                const long k = sa_koff(c, a.Vp) + (d - c8);
                float mv[8], pv[8];
#pragma unroll
                for (int x = 0; x < 8; ++x) {
                    const long dx = d + x;
                    const float tcdv = tcd[rr][8 * g + x], tdcv = tdc[8 * g + x][rr];
                    const bool valid = dx < a.V && dx >= c;
                    mv[x] = valid ? 0.5f * (tcdv - tdcv) : 0.0f;
                    pv[x] = !valid ? 0.0f : dx == c ? 0.5f * tcdv : 0.5f * (tcdv + tdcv);
                }
                // Am rows: the same-spin pairs, then the alpha-beta rows
                const long offM = (k >> 6) * a.rowsM * 64 + src * 64 + (k & 63);
                for (int sg = 0; sg < a.nseg; ++sg) {
                    uint32_t w4[4];
#pragma unroll
                    for (int x = 0; x < 4; ++x)
                        w4[x] = (uint32_t)__bfloat16_as_ushort(split_part(mv[2 * x], a.pat[sg])) |
                                ((uint32_t)__bfloat16_as_ushort(split_part(mv[2 * x + 1], a.pat[sg])) << 16);
                    *(uint4*)(a.Am + offM + sg * a.rowsM * a.Kp) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
                if (!ss) {
                    const long rowP = src - a.P2;
                    const long offP = (k >> 6) * a.rowsP * 64 + rowP * 64 + (k & 63);
                    for (int sg = 0; sg < a.nseg; ++sg) {
                        uint32_t w4[4];
#pragma unroll
                        for (int x = 0; x < 4; ++x)
                            w4[x] = (uint32_t)__bfloat16_as_ushort(split_part(pv[2 * x], a.pat[sg])) |
                                    ((uint32_t)__bfloat16_as_ushort(split_part(pv[2 * x + 1], a.pat[sg])) << 16);
                        *(uint4*)(a.Ap + offP + sg * a.rowsP * a.Kp) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// operand packing: strided FP64 view -> BF16 [rows][nseg * Kp] (K-major)
// ---------------------------------------------------------------------------
struct PackArgs {
    const double* src;
    __nv_bfloat16* dst;
    long rows, K, Kp;
    long ldd, segs;  // destination row pitch and segment stride (elements)
    long kbs;        // > 0: K-blocked destination, (r, k) at (k / 64) * kbs + r * 64 + k % 64
    int nseg;
    int pat[6];
    int nr, nk;
    long r_size[kMaxMode], r_s[kMaxMode];
    long k_size[kMaxMode], k_s[kMaxMode];
    int kfast;  // source contiguous along k
    long rvalid, kvalid;  // innermost row / k mode indices >= these read as 0
    const long* rtab;     // if set: row -> source offset (replaces the row modes)
    // Row modes are listed in the order tiles enumerate them (last fastest);
    // r_d is each mode's stride in the packed row index and rv_pos the mode
    // that rvalid applies to.
    long r_d[kMaxMode];
    int rv_pos;
};

// TR rows x TK k per tile (TR * TK = 4096): coalesced FP64 reads along
// whichever of row or k is contiguous in the source, conversion to FP32 in
// shared memory, then 16-byte stores of 8 BF16 values per segment.
template <int TR, int TK>
__global__ void __launch_bounds__(256) k_pack(PackArgs a) {
    __shared__ float tile[TR][TK + 1];
    __shared__ long roff[TR], rdst[TR], koff[TK];
    const long ntr = (a.rows + TR - 1) / TR, ntk = (a.Kp + TK - 1) / TK;
    const long ldd = a.ldd;
    for (long t = blockIdx.x; t < ntr * ntk; t += gridDim.x) {
        // consecutive tiles: along k for k-contiguous sources, along the rows
        // otherwise, so that the blocks in flight read nearby addresses (for
        // row-contiguous sources the k planes can be megabytes apart)
        const long r0 = (a.kfast ? t / ntk : t % ntr) * TR, k0 = (a.kfast ? t % ntk : t / ntr) * TK;
        // source offsets of the tile's rows and columns (-1: reads as zero)
        for (int x = threadIdx.x; x < TR + TK; x += blockDim.x) {
            if (x < TR) {
                const long r = r0 + x;
                long o = -1, d = -1;
                if (r < a.rows) {
                    if (a.rtab) {
                        o = a.rtab[r];
                        d = r;
                    } else {
                        unsigned u = (unsigned)r;
                        long so = 0, dr = 0;
                        bool ok = true;
#pragma unroll
                        for (int j = kMaxMode - 1; j >= 0; --j) {
                            if (j < a.nr) {
                                const unsigned sz = (unsigned)a.r_size[j];
                                const unsigned qq = u / sz, ix = u - qq * sz;
                                so += (long)ix * a.r_s[j];
                                dr += (long)ix * a.r_d[j];
                                if (j == a.rv_pos && (long)ix >= a.rvalid) ok = false;
                                u = qq;
                            }
                        }
                        d = dr;
                        if (ok) o = so;
                    }
                }
                roff[x] = o;
                rdst[x] = d;
            } else {
                const int kk = x - TR;
                const long k = k0 + kk;
                long o = -1;
                if (k < a.K) {
                    const unsigned ku = (unsigned)k;
                    if (a.nk == 0 || (long)(ku % (unsigned)a.k_size[a.nk - 1]) < a.kvalid)
                        o = decomp1_u32(ku, a.nk, a.k_size, a.k_s);
                }
                koff[kk] = o;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int e = threadIdx.x; e < TR * TK; e += 256) {
            int rr, kk;
            if (a.kfast) { kk = e % TK; rr = e / TK; }
            else { rr = e % TR; kk = e / TR; }
            const long ro = roff[rr], ko = koff[kk];
            tile[rr][kk] = (ro >= 0 && ko >= 0) ? f64_to_f32(a.src[ro + ko]) : 0.0f;
        }
        __syncthreads();
        // TR rows x TK/8 groups of 8 k
        constexpr int G = TK / 8;
        for (int it = threadIdx.x; it < TR * G; it += 256) {
            const int g = it % G, rr = it / G;
            const long r = rdst[rr];
            if (r < 0) continue;
            float v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = tile[rr][g * 8 + q];
            __nv_bfloat16* d = a.kbs > 0 ? a.dst + (k0 / 64) * a.kbs + r * 64 + g * 8 : a.dst + r * ldd + k0 + g * 8;
            for (int sg = 0; sg < a.nseg; ++sg) {
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    w[q] = (uint32_t)__bfloat16_as_ushort(split_part(v[2 * q], a.pat[sg])) |
                           ((uint32_t)__bfloat16_as_ushort(split_part(v[2 * q + 1], a.pat[sg])) << 16);
                *(uint4*)(d + (long)sg * a.segs) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        __syncthreads();
    }
}

// 8 consecutive BF16 values from element e0 of a 16-byte aligned array that
// extends to the next multiple of 8 elements past them: one aligned 16-byte
// load, or two and a shift by e0 % 8 elements
__device__ __forceinline__ uint4 load8_bf16(const uint16_t* base, long e0) {
    const int m = (int)(e0 & 7);
    const uint4* p = (const uint4*)(base + (e0 - m));
    const uint4 A = p[0];
    if (m == 0) return A;
    const uint4 B = p[1];
    const uint32_t w[8] = {A.x, A.y, A.z, A.w, B.x, B.y, B.z, B.w};
    const int h = m >> 1;
    uint32_t o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t lo = h == 0 ? w[q] : h == 1 ? w[q + 1] : h == 2 ? w[q + 2] : w[q + 3];
        const uint32_t hi = h == 0 ? w[q + 1] : h == 1 ? w[q + 2] : h == 2 ? w[q + 3] : w[q + 4];
        o[q] = (m & 1) ? __funnelshift_r(lo, hi, 16) : lo;
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
}

// The same packing from the BF16 image of the source (plane p = split part
// p of every element, planes `plane` elements apart): the parts are copied,
// so the packed operand is identical to the one k_pack makes from FP64.
// For sources with a unit-stride row mode (enumerated fastest): eight
// consecutive rows of one k that form one run of that mode are read as one
// 16-byte load (load8_bf16) and spread over the tile in shared memory.
// img points at the source's first element in plane 0 (img - imgbase is the
// plane's start, 16-byte aligned).
template <int TR, int TK>
__global__ void __launch_bounds__(256) k_pack_img(PackArgs a, const uint16_t* img, long plane, int nplanes,
                                                  long imgbase) {
    static_assert(TR % 8 == 0, "row groups of 8");
    __shared__ uint16_t tile[3][TR][TK + 2];
    __shared__ long roff[TR], rdst[TR], koff[TK];
    __shared__ int rrun[TR / 8];
    const long ntr = (a.rows + TR - 1) / TR, ntk = (a.Kp + TK - 1) / TK;
    const long ldd = a.ldd;
    const int np = nplanes < 3 ? nplanes : 3;
    for (long t = blockIdx.x; t < ntr * ntk; t += gridDim.x) {
        const long r0 = (a.kfast ? t / ntk : t % ntr) * TR, k0 = (a.kfast ? t % ntk : t / ntr) * TK;
        for (int x = threadIdx.x; x < TR + TK; x += blockDim.x) {
            if (x < TR) {
                const long r = r0 + x;
                long o = -1, d = -1;
                if (r < a.rows) {
                    if (a.rtab) {
                        o = a.rtab[r];
                        d = r;
                    } else {
                        unsigned u = (unsigned)r;
                        long so = 0, dr = 0;
                        bool ok = true;
#pragma unroll
                        for (int j = kMaxMode - 1; j >= 0; --j) {
                            if (j < a.nr) {
                                const unsigned sz = (unsigned)a.r_size[j];
                                const unsigned qq = u / sz, ix = u - qq * sz;
                                so += (long)ix * a.r_s[j];
                                dr += (long)ix * a.r_d[j];
                                if (j == a.rv_pos && (long)ix >= a.rvalid) ok = false;
                                u = qq;
                            }
                        }
                        d = dr;
                        if (ok) o = so;
                    }
                }
                roff[x] = o;
                rdst[x] = d;
            } else {
                const int kk = x - TR;
                const long k = k0 + kk;
                long o = -1;
                if (k < a.K) {
                    const unsigned ku = (unsigned)k;
                    if (a.nk == 0 || (long)(ku % (unsigned)a.k_size[a.nk - 1]) < a.kvalid)
                        o = decomp1_u32(ku, a.nk, a.k_size, a.k_s);
                }
                koff[kk] = o;
            }
        }
        __syncthreads();
        if (threadIdx.x < TR / 8) {
            const int g = threadIdx.x;
            int run = !a.kfast && roff[8 * g] >= 0;
            for (int q = 1; q < 8 && run; ++q) run = roff[8 * g + q] == roff[8 * g] + q;
            rrun[g] = run;
        }
        __syncthreads();
        if (!a.kfast) {
            // consecutive threads: consecutive row groups of one k
            for (int e = threadIdx.x; e < (TR / 8) * TK; e += 256) {
                const int g = e % (TR / 8), kk = e / (TR / 8);
                const long ko = koff[kk];
                if (ko >= 0 && rrun[g]) {
                    for (int p = 0; p < np; ++p) {
                        const uint4 v = load8_bf16(img - imgbase + p * plane, imgbase + roff[8 * g] + ko);
                        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int q = 0; q < 8; ++q) tile[p][8 * g + q][kk] = (uint16_t)(w[q >> 1] >> (16 * (q & 1)));
                    }
                } else {
                    for (int q = 0; q < 8; ++q) {
                        const long ro = roff[8 * g + q];
                        const bool in = ro >= 0 && ko >= 0;
                        for (int p = 0; p < np; ++p) tile[p][8 * g + q][kk] = in ? img[p * plane + ro + ko] : (uint16_t)0;
                    }
                }
            }
        } else {
#pragma unroll 4
            for (int e = threadIdx.x; e < TR * TK; e += 256) {
                const int kk = e % TK, rr = e / TK;
                const long ro = roff[rr], ko = koff[kk];
                const bool in = ro >= 0 && ko >= 0;
                for (int p = 0; p < np; ++p) tile[p][rr][kk] = in ? img[p * plane + ro + ko] : (uint16_t)0;
            }
        }
        __syncthreads();
        constexpr int G = TK / 8;
        for (int it = threadIdx.x; it < TR * G; it += 256) {
            const int g = it % G, rr = it / G;
            const long r = rdst[rr];
            if (r < 0) continue;
            __nv_bfloat16* d = a.kbs > 0 ? a.dst + (k0 / 64) * a.kbs + r * 64 + g * 8 : a.dst + r * ldd + k0 + g * 8;
            for (int sg = 0; sg < a.nseg; ++sg) {
                const uint16_t* v = &tile[a.pat[sg]][rr][g * 8];
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) w[q] = (uint32_t)v[2 * q] | ((uint32_t)v[2 * q + 1] << 16);
                *(uint4*)(d + (long)sg * a.segs) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        __syncthreads();
    }
}

// Packing from the BF16 image of a source contiguous along its innermost k
// mode (rows in packed order): one warp per (row, 2048 consecutive k), eight
// k per lane and step.  The row offset is decomposed once per item and the
// k mode indices are advanced, not recomputed.  Eight k inside one run of the
// innermost mode are one 16-byte read (load8_bf16), others are gathered one
// by one; each segment leaves as one 16-byte store.  img: the source's first
// element in plane 0 (plane p = part p, `plane` elements further); imgbase:
// its element index in the plane (img - imgbase: the plane's aligned start).
__global__ void __launch_bounds__(256) k_pack_rows_img(PackArgs a, const uint16_t* img, long plane, int nplanes,
                                                       long imgbase) {
    constexpr long KCH = 2048;
    const int lane = threadIdx.x & 31;
    const long nkc = (a.Kp + KCH - 1) / KCH;
    const long nitems = a.rows * nkc;
    const long wstride = (long)gridDim.x * (blockDim.x >> 5);
    const int nk = a.nk;
    const long kin = nk > 0 ? a.k_size[nk - 1] : 1;
    const bool unit = nk > 0 && a.k_s[nk - 1] == 1;
    const int np = nplanes < 3 ? nplanes : 3;
    int used = 0;
    for (int sg = 0; sg < a.nseg; ++sg) used |= 1 << a.pat[sg];
    for (long w = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nitems; w += wstride) {
        const long r = w / nkc, kb = (w - r * nkc) * KCH, ke = kb + KCH < a.Kp ? kb + KCH : a.Kp;
        long ro = -1;
        if (a.rtab) {
            ro = a.rtab[r];
        } else {
            unsigned u = (unsigned)r;
            long so = 0;
            bool ok = true;
#pragma unroll
            for (int j = kMaxMode - 1; j >= 0; --j) {
                if (j < a.nr) {
                    const unsigned sz = (unsigned)a.r_size[j];
                    const unsigned qq = u / sz, ix = u - qq * sz;
                    so += (long)ix * a.r_s[j];
                    if (j == a.rv_pos && (long)ix >= a.rvalid) ok = false;
                    u = qq;
                }
            }
            if (ok) ro = so;
        }
        long k0 = kb + 8 * lane;
        long idx[kMaxMode];
        {
            unsigned u = (unsigned)(k0 < a.K ? k0 : 0);
#pragma unroll
            for (int j = kMaxMode - 1; j >= 0; --j) {
                idx[j] = 0;
                if (j < nk) {
                    const unsigned sz = (unsigned)a.k_size[j];
                    const unsigned qq = u / sz;
                    idx[j] = (long)(u - qq * sz);
                    u = qq;
                }
            }
        }
        for (; k0 < ke; k0 += 256) {
            long off = 0;
#pragma unroll
            for (int j = 0; j < kMaxMode; ++j)
                if (j < nk) off += idx[j] * a.k_s[j];
            const long in0 = nk > 0 ? idx[nk - 1] : 0;
            const bool run = ro >= 0 && unit && k0 + 8 <= a.K && in0 + 8 <= kin && in0 + 8 <= a.kvalid;
            uint4 v[3] = {};
            if (run) {
                for (int p = 0; p < np; ++p)
                    if (used & (1 << p)) v[p] = load8_bf16(img - imgbase + p * plane, imgbase + ro + off);
            } else {
                uint32_t wv[3][4] = {};
                long id[kMaxMode];
#pragma unroll
                for (int j = 0; j < kMaxMode; ++j) id[j] = idx[j];
                for (int q = 0; q < 8; ++q) {
                    const long k = k0 + q;
                    if (ro >= 0 && k < a.K && (nk == 0 || id[nk - 1] < a.kvalid)) {
                        long o = ro;
#pragma unroll
                        for (int j = 0; j < kMaxMode; ++j)
                            if (j < nk) o += id[j] * a.k_s[j];
                        for (int p = 0; p < np; ++p)
                            if (used & (1 << p)) wv[p][q >> 1] |= (uint32_t)img[p * plane + o] << (16 * (q & 1));
                    }
                    for (int j = nk - 1; j >= 0; --j) {
                        if (++id[j] < a.k_size[j]) break;
                        id[j] = 0;
                    }
                }
                for (int p = 0; p < 3; ++p) v[p] = make_uint4(wv[p][0], wv[p][1], wv[p][2], wv[p][3]);
            }
            __nv_bfloat16* d = a.kbs > 0 ? a.dst + (k0 / 64) * a.kbs + r * 64 + (k0 & 63) : a.dst + r * a.ldd + k0;
            for (int sg = 0; sg < a.nseg; ++sg) *(uint4*)(d + (long)sg * a.segs) = v[a.pat[sg]];
            // the mode indices of k0 + 256 (innermost first, carries outward)
            if (nk > 0 && k0 + 256 < a.K) {
                idx[nk - 1] += 256;
                for (int j = nk - 1; j > 0; --j) {
                    if (idx[j] < a.k_size[j]) break;
                    const long qq = idx[j] / a.k_size[j];
                    idx[j] -= qq * a.k_size[j];
                    idx[j - 1] += qq;
                }
            }
        }
    }
}

// plane p of the image = part p of the split of every element (as k_pack
// computes it: FP64 -> FP32, then hi, mid, lo)
__global__ void k_t2_image(const double* __restrict__ t2, long n, long plane, int nplanes, uint16_t* __restrict__ img) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; 2 * i < n; i += (long)gridDim.x * blockDim.x) {
        if (2 * i + 1 < n) {
            const double2 v = *(const double2*)(t2 + 2 * i);
            const float x0 = f64_to_f32(v.x), x1 = f64_to_f32(v.y);
            for (int p = 0; p < nplanes; ++p)
                *(uint32_t*)(img + p * plane + 2 * i) = (uint32_t)__bfloat16_as_ushort(split_part(x0, p)) |
                                                          ((uint32_t)__bfloat16_as_ushort(split_part(x1, p)) << 16);
        } else {
            const float x0 = f64_to_f32(t2[2 * i]);
            for (int p = 0; p < nplanes; ++p) img[p * plane + 2 * i] = __bfloat16_as_ushort(split_part(x0, p));
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Buf {
    __nv_bfloat16* p = nullptr;
    size_t cap = 0;  // elements
};

struct TcEngine {
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    int* d_err = nullptr;
    int mc_clusters[2] = {0, 0};  // resident two-CTA clusters (BN 128, 256); 0 unknown, -1 none
    Buf pa, pb, pv, pt;  // generic A, generic B, ladder V tile, stacked amplitudes
    bool attr_set = false;
    // ladder row tables for the stacked amplitudes [aa pairs; bb pairs; ab; ab~]
    long tab_O = -1, tab_V = -1;
    long* d_pairoff = nullptr;  // [2P] t2 offset of the same-spin pair rows
    int* d_rowcode = nullptr;   // [rows] block/i/j code of every row
    long* d_growoff = nullptr;  // [rows] offset of the row's G[blk][i][j] slice
    float* wsk = nullptr;       // split-K partial tiles
    size_t wsk_cap = 0;
    static constexpr int kPackSlots = 4;
    Buf pc[kPackSlots];         // pack cache (see pack_operand)
    std::string pc_key[kPackSlots];
    long pc_tick[kPackSlots] = {};
    long pc_clock = 0;
    // symmetric / antisymmetric ladder: amplitudes A- (same-spin pairs and
    // alpha-beta rows) and A+ (alpha-beta rows), the M+ and M- tiles of a
    // chunk, the DF factors packed [(x, y)][L] with the A- and B-side split
    // patterns, and the consumer row codes
    Buf sam, sap, svp, svm, sxa, sxb;
    int* d_code_m = nullptr;
    int* d_code_p = nullptr;
    long sa_O = -1;
    bool sa_attr = false;
    int sx_nsplit = 0;  // split of the packed DF factors in sxa / sxb (0: none; B never changes)
    // packed operands read from the DF factors B or from J, which never
    // change after initialisation: kept for the life of the context (key as
    // in pack_operand), up to kBCacheBytes in all
    static constexpr size_t kBCacheBytes = 8ul << 30;
    std::vector<std::pair<std::string, Buf>> bcache;
    size_t bcache_bytes = 0;
    Buf pbv;            // the ladder's B_vv [(b,d)][L] for the G pass
    int pbv_nsplit = 0; // its split (0: not packed)
};

static dcsd_status ensure(Ctx* c, Buf& b, size_t elems) {
    if (b.cap >= elems) return DCSD_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (cudaMalloc((void**)&b.p, elems * sizeof(__nv_bfloat16)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "cudaMalloc of BF16 operand buffer failed";
        return DCSD_ERR_OOM;
    }
    b.cap = elems;
    return DCSD_OK;
}

dcsd_status tc_init(Ctx* c) {
    TcEngine* e = new TcEngine();
    c->tc = e;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        c->err = "cuTensorMapEncodeTiled unavailable";
        return DCSD_ERR_CUDA;
    }
    e->encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    e->d_err = (int*)(c->scal + 22);  // device error word, read back with the scalars
    DCSD_CUDA(c, cudaMemset(c->scal, 0, 64 * sizeof(double)));
    return DCSD_OK;
}

void tc_free(Ctx* c) {
    TcEngine* e = c->tc;
    if (!e) return;
    for (Buf* b : {&e->pa, &e->pb, &e->pv, &e->pt, &e->sam, &e->sap, &e->svp, &e->svm, &e->sxa, &e->sxb, &e->pbv})
        if (b->p) cudaFree(b->p);
    for (auto& kv : e->bcache)
        if (kv.second.p) cudaFree(kv.second.p);
    if (e->d_code_m) cudaFree(e->d_code_m);
    if (e->d_code_p) cudaFree(e->d_code_p);
    if (e->d_pairoff) cudaFree(e->d_pairoff);
    if (e->d_rowcode) cudaFree(e->d_rowcode);
    if (e->d_growoff) cudaFree(e->d_growoff);
    if (e->wsk) cudaFree(e->wsk);
    for (auto& b : e->pc)
        if (b.p) cudaFree(b.p);
    delete e;
    c->tc = nullptr;
}

static long round_up(long x, long m) { return (x + m - 1) / m * m; }

// K-major operand [rows][pitch] (BF16), of which the first kt columns are
// read (pitch 0: kt); p and pitch * 2 bytes must be 16-byte aligned
static dcsd_status make_map(Ctx* c, CUtensorMap* map, const __nv_bfloat16* p, long rows, long kt,
                            int box_rows, long pitch = 0) {
    if (pitch == 0) pitch = kt;
    cuuint64_t dims[2] = {(cuuint64_t)kt, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(pitch * 2)};
    cuuint32_t box[2] = {TC_BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = c->tc->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)p, dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
        return DCSD_ERR_CUDA;
    }
    return DCSD_OK;
}

// Packs rows x K (padded to Kp) of a strided FP64 source into nseg BF16
// split segments.  Element (row r, segment s, k) goes to
// dst[r * ldd + s * segs + k]; the defaults (ldd = nseg * Kp, segs = Kp) put
// a row's segments side by side, segs = rows_total * Kp with ldd = Kp keeps
// each segment a contiguous [rows][Kp] operand; kbs > 0 (with segs) stores
// each segment K-blocked, (r, k) at (k / 64) * kbs + r * 64 + k % 64.
static dcsd_status pack(Ctx* c, const double* src, int nr, const long* rsz, const long* rs, int nk,
                        const long* ksz, const long* ks, long rows, long K, long Kp, int nseg,
                        const int* pat, __nv_bfloat16* dst, long rvalid = 1l << 62,
                        long kvalid = 1l << 62, const long* rtab = nullptr, long ldd = 0, long segs = 0,
                        long kbs = 0) {
    PackArgs a;
    a.ldd = ldd > 0 ? ldd : (long)nseg * Kp;
    a.segs = segs > 0 ? segs : Kp;
    a.kbs = kbs;
    a.rtab = rtab;
    a.rvalid = rvalid;
    a.kvalid = kvalid;
    a.src = src;
    a.dst = dst;
    a.rows = rows;
    a.K = K;
    a.Kp = Kp;
    a.nseg = nseg;
    for (int i = 0; i < 6; ++i) a.pat[i] = i < nseg ? pat[i] : 0;
    a.nr = nr;
    a.nk = nk;
    a.kfast = (nk > 0 && ks[nk - 1] == 1) ? 1 : 0;
    // enumeration order of the row modes: the packed order, except that a
    // source that is contiguous along a slower row mode (and not along k)
    // has that mode enumerated fastest, so each tile reads contiguous runs
    int order[kMaxMode];
    for (int i = 0; i < nr; ++i) order[i] = i;
    bool rowcontig = false;  // some row mode has unit stride
    for (int i = 0; i < nr && !rtab; ++i)
        if (std::labs(rs[i]) == 1 && rsz[i] > 1) rowcontig = true;
    if (!rtab && !a.kfast && nr >= 2) {
        int js = -1;
        for (int i = 0; i < nr; ++i)
            if (std::labs(rs[i]) == 1 && rsz[i] > 1) js = i;
        if (js >= 0 && js != nr - 1) {
            for (int i = js; i < nr - 1; ++i) order[i] = order[i + 1];
            order[nr - 1] = js;
        }
    }
    long dstr[kMaxMode];
    long st = 1;
    for (int i = nr - 1; i >= 0; --i) {
        dstr[i] = st;
        st *= rsz[i];
    }
    a.rv_pos = -1;
    for (int i = 0; i < kMaxMode; ++i) {
        a.r_size[i] = i < nr ? rsz[order[i]] : 1;
        a.r_s[i] = i < nr ? rs[order[i]] : 0;
        a.r_d[i] = i < nr ? dstr[order[i]] : 0;
        if (i < nr && order[i] == nr - 1) a.rv_pos = i;
        a.k_size[i] = i < nk ? ksz[i] : 1;
        a.k_s[i] = i < nk ? ks[i] : 0;
    }
    if (Kp % 64 != 0 || rows >= (1l << 31) || Kp >= (1l << 31)) {
        c->err = "pack: K padding must be a multiple of 64 and sizes below 2^31";
        return DCSD_ERR_INVALID_ARG;
    }
    const int TR = 64, TK = 64;
    long tiles = ((rows + TR - 1) / TR) * (Kp / TK);
    unsigned g = (unsigned)std::max<long>(1, std::min<long>(tiles, (long)c->num_sms * 8));
    // a view of t2 while its BF16 image holds every part the segments use:
    // copy the parts from the image (the same offsets address it)
    const uint16_t* img = nullptr;
    if (!c->pack_generic && c->t2img_src && src >= c->t2img_src && src < c->t2img_src + c->t2img_len) {
        img = c->t2img + (src - c->t2img_src);
        for (int i = 0; i < nseg; ++i)
            if (pat[i] < 0 || pat[i] >= c->t2img_planes) img = nullptr;
    }
    prof_begin(c, DCSD_PROF_PACK);
    if (c->trace) {
        const std::string label = "pack " + c->cur_spec + " rows=" + std::to_string(rows) + " K=" + std::to_string(K) +
                                  " kfast=" + std::to_string(a.kfast) + (img && (a.kfast || rowcontig) ? " img" : "");
        if (c->trace_seq) fprintf(stderr, "[dcsd pack #%d] %s\n", c->pack_seq, label.c_str());
        trace_begin(c, label);
    }
    ++c->pack_seq;
    if (img && a.kfast) {
        // rows in packed order, source contiguous along k: warp per row run
        const long items = rows * ((Kp + 2047) / 2048);
        const unsigned gr = (unsigned)std::max<long>(1, std::min<long>((items + 7) / 8, (long)c->num_sms * 16));
        k_pack_rows_img<<<gr, 256, 0, c->stream>>>(a, img, c->t2img_plane, c->t2img_planes,
                                                    (long)(src - c->t2img_src));
    } else if (img && rowcontig) {
        // (without a unit-stride row mode the tile's reads are scattered,
        // and 2-byte reads waste more of each sector than 8-byte ones)
        k_pack_img<64, 64><<<g, 256, 0, c->stream>>>(a, img, c->t2img_plane, c->t2img_planes,
                                                     (long)(src - c->t2img_src));
    } else {
        k_pack<64, 64><<<g, 256, 0, c->stream>>>(a);
    }
    trace_end(c);
    prof_end(c, DCSD_PROF_PACK);
    return launch_check(c, "tc_pack");
}

// C = alpha * A_p B_p^T (+ beta C); A_p [M][Ktot], B_p [N][Ktot] packed BF16
// K-blocked operand [kt / 64][rows][64] (BF16): one TMA box of box_rows rows
// and 64 k is a contiguous block of memory
static dcsd_status make_map_kblk(Ctx* c, CUtensorMap* map, const __nv_bfloat16* p, long rows, long kt,
                                 int box_rows) {
    cuuint64_t dims[3] = {(cuuint64_t)TC_BK, (cuuint64_t)rows, (cuuint64_t)(kt / TC_BK)};
    cuuint64_t strides[2] = {(cuuint64_t)(TC_BK * 2), (cuuint64_t)(rows * TC_BK * 2)};
    cuuint32_t box[3] = {TC_BK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = c->tc->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)p, dims, strides, box, es,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->err = "cuTensorMapEncodeTiled (K-blocked) failed (" + std::to_string((int)r) + ")";
        return DCSD_ERR_CUDA;
    }
    return DCSD_OK;
}

// C (epilogue epi) = A[M][Ktot] . B[N][Ktot]^T; the operands are K-major BF16
// with row pitch `pitch` elements (0: Ktot), or K-blocked (kblocked: both
// operands [Ktot / 64][rows][64])
// mc (K-blocked operands, at least two m-tiles): clusters of two CTAs share
// each B tile through TMA multicast (see k_tc_gemm)
static dcsd_status gemm_packed(Ctx* c, const __nv_bfloat16* Ap, long M, const __nv_bfloat16* Bp, long N,
                               long Ktot, TcEpi& epi, int ksplit = 1, long pitch = 0, bool kblocked = false,
                               bool mc = false) {
    TcEngine* e = c->tc;
    if (!e->attr_set) {
        size_t s256 = TC_STAGES * (TC_BM * TC_BK * 2 + 256 * TC_BK * 2) + kStageBytesMode2 + 2048;
        size_t s128 = TC_STAGES * (TC_BM * TC_BK * 2 + 128 * TC_BK * 2) + kStageBytesMode2 + 2048;
        DCSD_CUDA(c, cudaFuncSetAttribute(k_tc_gemm<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)s256));
        DCSD_CUDA(c, cudaFuncSetAttribute(k_tc_gemm<128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)s128));
        DCSD_CUDA(c, cudaFuncSetAttribute(k_tc_gemm<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)s256));
        DCSD_CUDA(c, cudaFuncSetAttribute(k_tc_gemm<128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)s128));
        e->attr_set = true;
    }
    const int BN = N >= 256 ? 256 : 128;
    mc = mc && kblocked && c->tc_multicast && M > TC_BM && c->num_sms >= 2;
    long max_clusters = c->num_sms / 2;
    if (mc) {
        if (e->mc_clusters[BN == 256 ? 1 : 0] == 0) {
            cudaLaunchConfig_t q = {};
            q.gridDim = dim3((unsigned)(2 * max_clusters));
            q.blockDim = dim3(kTcThreads);
            q.dynamicSmemBytes = TC_STAGES * (TC_BM * TC_BK * 2 + (size_t)BN * TC_BK * 2) + kStageBytesMode2 + 2048;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            q.attrs = at;
            q.numAttrs = 1;
            int nclu = 0;
            const cudaError_t qe = BN == 256 ? cudaOccupancyMaxActiveClusters(&nclu, k_tc_gemm<256, true>, &q)
                                             : cudaOccupancyMaxActiveClusters(&nclu, k_tc_gemm<128, true>, &q);
            if (qe != cudaSuccess || nclu < 1) {
                cudaGetLastError();
                nclu = -1;  // clusters unavailable: the one-CTA kernel runs
            }
            e->mc_clusters[BN == 256 ? 1 : 0] = nclu;
        }
        const int nclu = e->mc_clusters[BN == 256 ? 1 : 0];
        if (nclu < 1) mc = false;
        else max_clusters = std::min<long>(max_clusters, nclu);
    }
    CUtensorMap ma, mb;
    if (pitch != 0 && (pitch < Ktot || pitch % 8 != 0 || ((uintptr_t)Ap | (uintptr_t)Bp) % 16 != 0)) {
        c->err = "tensor-core GEMM: operand pitch or base not aligned";
        return DCSD_ERR_INVALID_ARG;
    }
    if (kblocked) {
        if (Ktot % TC_BK != 0 || ((uintptr_t)Ap | (uintptr_t)Bp) % 16 != 0) {
            c->err = "tensor-core GEMM: K-blocked operands need K % 64 == 0 and 16-byte aligned bases";
            return DCSD_ERR_INVALID_ARG;
        }
        DCSD_TRY(make_map_kblk(c, &ma, Ap, M, Ktot, TC_BM));
        DCSD_TRY(make_map_kblk(c, &mb, Bp, N, Ktot, mc ? BN / 2 : BN));
    } else {
        DCSD_TRY(make_map(c, &ma, Ap, M, Ktot, TC_BM, pitch));
        DCSD_TRY(make_map(c, &mb, Bp, N, Ktot, BN, pitch));
    }
    epi.M = M;
    epi.N = N;
    const int nkt = (int)(Ktot / TC_BK);
    const long tilesM = (M + TC_BM - 1) / TC_BM, tilesN = (N + BN - 1) / BN;
    if (tilesM * tilesN > (1l << 31) - 1 || M >= (1l << 31) || N >= (1l << 31)) {
        c->err = "tensor-core GEMM too large";
        return DCSD_ERR_INVALID_ARG;
    }
    ksplit = std::max(1, std::min(ksplit, nkt));
    const int kper = (nkt + ksplit - 1) / ksplit;
    const long ntiles = tilesM * tilesN * ((nkt + kper - 1) / kper);
    if (ntiles > (1l << 31) - 1) {
        c->err = "tensor-core GEMM too large";
        return DCSD_ERR_INVALID_ARG;
    }
    // MC: the schedule runs over pairs of m-tiles, two CTAs per pair; as many
    // clusters as can be resident at once (a persistent grid)
    const long tilesMs = mc ? (tilesM + 1) / 2 : tilesM;
    const long ntiles_s = tilesMs * tilesN * ((nkt + kper - 1) / kper);
    dim3 grid((unsigned)(mc ? 2 * std::min<long>(ntiles_s, max_clusters) : std::min<long>(ntiles, c->num_sms)));
    // m-tile band height that minimises the A and B rows one wave of
    // num_sms tiles touches: g * BM + (num_sms / g) * BN
    // (an operand that fits in a quarter of L2 is kept there instead: all
    // m-tiles of a band when A fits, one m-tile per band when B fits)
    int group = (int)std::lround(std::sqrt((double)c->num_sms * BN / TC_BM));
    const double l2q = 32e6;
    // (the ladder's long-K contractions measured best with all m-tiles per band)
    if ((double)M * (double)Ktot * 2.0 <= l2q || c->ladder_phase) group = (int)tilesM;
    else if ((double)N * (double)Ktot * 2.0 <= l2q) group = 1;
    group = (int)std::max<long>(1, std::min<long>(group, tilesM));
    if (mc) group = (int)std::max<long>(1, std::min<long>((group + 1) / 2, tilesMs));
    size_t smem = TC_STAGES * (TC_BM * TC_BK * 2 + (size_t)BN * TC_BK * 2) + kStageBytesMode2 + 2048;
    const int cls = c->ladder_phase ? DCSD_PROF_LADDER : DCSD_PROF_TC_OTHER;
    prof_begin(c, cls);
    if (c->trace) {
        const std::string label = std::string(c->ladder_phase ? "tc-ladder " : "tc ") + c->cur_spec +
                                  " mode=" + std::to_string(epi.mode) + " M=" + std::to_string(M) +
                                  " N=" + std::to_string(N) + " Kt=" + std::to_string(Ktot);
        if (c->trace_seq) fprintf(stderr, "[dcsd tc #%d] %s\n", c->tc_seq, label.c_str());
        trace_begin(c, label);
    }
    ++c->tc_seq;
    if (mc) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(kTcThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const int tm = (int)tilesM, tn = (int)tilesN, kb = 1;
        cudaError_t le = BN == 256 ? cudaLaunchKernelEx(&cfg, k_tc_gemm<256, true>, ma, mb, epi, nkt, tm, tn, kper, group,
                                                        kb, e->d_err)
                                   : cudaLaunchKernelEx(&cfg, k_tc_gemm<128, true>, ma, mb, epi, nkt, tm, tn, kper, group,
                                                        kb, e->d_err);
        if (le != cudaSuccess) {
            trace_end(c);
            prof_end(c, cls);
            c->err = std::string("tc_gemm (cluster launch): ") + cudaGetErrorString(le);
            cudaGetLastError();
            return DCSD_ERR_CUDA;
        }
    } else if (BN == 256) {
        k_tc_gemm<256, false><<<grid, kTcThreads, smem, c->stream>>>(ma, mb, epi, nkt, (int)tilesM, (int)tilesN, kper,
                                                                     group, kblocked ? 1 : 0, e->d_err);
    } else {
        k_tc_gemm<128, false><<<grid, kTcThreads, smem, c->stream>>>(ma, mb, epi, nkt, (int)tilesM, (int)tilesN, kper,
                                                                     group, kblocked ? 1 : 0, e->d_err);
    }
    trace_end(c);
    prof_end(c, cls);
    return launch_check(c, "tc_gemm");
}

dcsd_status einsum_tc_impl(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B, double beta,
                           const TV& C, int nsplit);

// Pack one operand into `dflt`, or, when its source is one of the context's
// pack-cache sources (set by callers that contract the same operands many
// times with unchanged data), reuse a cache slot holding the same packing
// (same source, modes, strides and split pattern) or repack into the least
// recently used slot.  The slot used by the other operand of the current
// contraction is the most recently used one, so it is never the one evicted.
static dcsd_status pack_operand(Ctx* c, const double* src, int nr, const long* rsz, const long* rs, int nk,
                                const long* ksz, const long* ks, long rows, long K, long Kp, int nseg,
                                const int* pat, Buf& dflt, const __nv_bfloat16*& out) {
    TcEngine* e = c->tc;
    bool cached = false;
    for (int k = 0; k < 2; ++k)
        if (src && src == c->pack_cache_src[k]) cached = true;
    // views of the DF factors B and of J = (kc|ld), both made at
    // initialisation and never changed: packed once for the life of the context
    const size_t nB = (size_t)c->X * c->n * c->n, nJ = (size_t)c->O * c->O * c->V * c->V;
    if (src && ((c->B && src >= c->B && src < c->B + nB) || (c->J && src >= c->J && src < c->J + nJ))) {
        std::string key = std::to_string((uintptr_t)src) + "|" + std::to_string(nr) + "|" + std::to_string(nk) + "|" +
                          std::to_string(rows) + "|" + std::to_string(K) + "|" + std::to_string(Kp) + "|" +
                          std::to_string(nseg);
        for (int i = 0; i < nr; ++i) key += "|r" + std::to_string(rsz[i]) + ":" + std::to_string(rs[i]);
        for (int i = 0; i < nk; ++i) key += "|k" + std::to_string(ksz[i]) + ":" + std::to_string(ks[i]);
        for (int i = 0; i < nseg; ++i) key += "|p" + std::to_string(pat[i]);
        for (auto& kv : e->bcache)
            if (kv.first == key) {
                out = kv.second.p;
                return DCSD_OK;
            }
        const size_t bytes = (size_t)rows * nseg * Kp * sizeof(__nv_bfloat16);
        if (e->bcache_bytes + bytes <= TcEngine::kBCacheBytes) {
            Buf b;
            DCSD_TRY(ensure(c, b, (size_t)rows * nseg * Kp));
            const dcsd_status st = pack(c, src, nr, rsz, rs, nk, ksz, ks, rows, K, Kp, nseg, pat, b.p);
            if (st != DCSD_OK) {
                cudaFree(b.p);
                return st;
            }
            e->bcache.push_back({key, b});
            e->bcache_bytes += bytes;
            out = b.p;
            return DCSD_OK;
        }
    }
    if (!cached) {
        DCSD_TRY(ensure(c, dflt, (size_t)rows * nseg * Kp));
        DCSD_TRY(pack(c, src, nr, rsz, rs, nk, ksz, ks, rows, K, Kp, nseg, pat, dflt.p));
        out = dflt.p;
        return DCSD_OK;
    }
    std::string key = std::to_string((uintptr_t)src) + "|" + std::to_string(nr) + "|" + std::to_string(nk) + "|" +
                      std::to_string(rows) + "|" + std::to_string(K) + "|" + std::to_string(Kp) + "|" +
                      std::to_string(nseg);
    for (int i = 0; i < nr; ++i) key += "|r" + std::to_string(rsz[i]) + ":" + std::to_string(rs[i]);
    for (int i = 0; i < nk; ++i) key += "|k" + std::to_string(ksz[i]) + ":" + std::to_string(ks[i]);
    for (int i = 0; i < nseg; ++i) key += "|p" + std::to_string(pat[i]);
    int slot = -1;
    for (int k = 0; k < TcEngine::kPackSlots; ++k)
        if (e->pc_key[k] == key) slot = k;
    if (slot < 0) {
        slot = 0;
        for (int k = 1; k < TcEngine::kPackSlots; ++k)
            if (e->pc_tick[k] < e->pc_tick[slot]) slot = k;
        e->pc_key[slot].clear();
        DCSD_TRY(ensure(c, e->pc[slot], (size_t)rows * nseg * Kp));
        DCSD_TRY(pack(c, src, nr, rsz, rs, nk, ksz, ks, rows, K, Kp, nseg, pat, e->pc[slot].p));
        e->pc_key[slot] = key;
    }
    e->pc_tick[slot] = ++e->pc_clock;
    out = e->pc[slot].p;
    return DCSD_OK;
}

dcsd_status t2_image(Ctx* c, int nsplit) {
    c->t2img_src = nullptr;
    const long n = 3 * c->O * c->O * c->V * c->V;
    const long plane = round_up(n, 8);
    const int np = std::max(1, std::min(3, nsplit));
    const size_t need = (size_t)np * plane;
    if (c->t2img_cap < need) {
        if (c->t2img) cudaFree(c->t2img);
        c->t2img = nullptr;
        c->t2img_cap = 0;
        DCSD_CUDA(c, cudaMalloc((void**)&c->t2img, need * sizeof(uint16_t)));
        c->t2img_cap = need;
    }
    if (c->trace) trace_begin(c, "t2 image planes=" + std::to_string(np));
    const long pairs = (n + 1) / 2;
    k_t2_image<<<(unsigned)std::max<long>(1, std::min<long>((pairs + 255) / 256, (long)c->num_sms * 16)), 256, 0,
                 c->stream>>>(c->t2, n, plane, np, c->t2img);
    trace_end(c);
    DCSD_TRY(launch_check(c, "t2_image"));
    c->t2img_src = c->t2;
    c->t2img_len = n;
    c->t2img_plane = plane;
    c->t2img_planes = np;
    return DCSD_OK;
}

void pack_cache_set(Ctx* c, const double* src0, const double* src1) {
    c->pack_cache_src[0] = src0;
    c->pack_cache_src[1] = src1;
    if (!c->tc) return;
    TcEngine* e = c->tc;
    for (int k = 0; k < TcEngine::kPackSlots; ++k) {
        e->pc_key[k].clear();
        e->pc_tick[k] = 0;
        // the slots hold up to a few GB each: released when the cache is cleared
        if (!src0 && !src1 && e->pc[k].p) {
            cudaFree(e->pc[k].p);
            e->pc[k] = Buf();
        }
    }
}

// Segments along K whose products sum to the split product:
//   nsplit 2: x = h + m;       hh + hm + mh                (3 BF16 products)
//   nsplit 3: x = h + m + l;   hh + hm + mh + hl + lh + mm (6 BF16 products)
static void split_patterns(int nsplit, int& nseg, int* pa, int* pb) {
    for (int i = 0; i < 6; ++i) pa[i] = pb[i] = 0;
    if (nsplit == 3) {
        nseg = 6;
        const int A[6] = {0, 0, 1, 0, 2, 1}, B[6] = {0, 1, 0, 2, 0, 1};
        for (int i = 0; i < 6; ++i) { pa[i] = A[i]; pb[i] = B[i]; }
    } else if (nsplit == 2) {
        nseg = 3;
        pa[0] = 0; pa[1] = 0; pa[2] = 1;  // A: h h m
        pb[0] = 0; pb[1] = 1; pb[2] = 0;  // B: h m h
    } else {
        nseg = 1;
    }
}

// C[m,n] = alpha * sum_s ws[(s * N + n) * M + m] (+ beta * C), or the FP32
// shadow += alpha * sum (mode 4), with the offsets of the epilogue's modes
__global__ void k_tc_splitk_reduce(TcEpi epi, int ksplit, const float* ws) {
    const long MN = epi.M * epi.N;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < MN; e += (long)gridDim.x * blockDim.x) {
        const long n = e / epi.M, m = e - n * epi.M;
        double v = 0.0;
        for (int s = 0; s < ksplit; ++s) v += (double)ws[(long)s * MN + e];
        const long off = decomp1(m, epi.nm, epi.m_size, epi.m_s) + decomp1(n, epi.nn, epi.n_size, epi.n_s);
        if (epi.mode == 4) {
            epi.C32[off] += (float)(epi.alpha * v);
        } else {
            const double r = epi.alpha * v;
            epi.C[off] = epi.beta != 0.0 ? fma(epi.beta, epi.C[off], r) : r;
        }
    }
}

dcsd_status einsum_tc(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B, double beta,
                      const TV& C, int nsplit) {
    const bool rec = c->rec;
    if (rec) {
        // one tape entry; the engine's own fallbacks are not recorded again
        record_einsum(c, spec, alpha, A, B, beta, C, 2, nsplit);
        c->rec = false;
    }
    c->cur_spec = spec;
    dcsd_status st = einsum_tc_impl(c, spec, alpha, A, B, beta, C, nsplit);
    c->cur_spec = c->ladder_phase ? "ladder" : "";
    c->rec = rec;
    return st;
}

// accuracy split of long BF16X6 contractions (at least 4 x 64 k-blocks):
// FP32 partials over <= 64 k-blocks (4096 products), when the partial tiles
// take at most 3 GB
constexpr long kAccBlocks = 64;
constexpr double kAccWorkspaceBytes = 3e9;

dcsd_status einsum_tc_impl(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B, double beta,
                           const TV& C, int nsplit) {
    GemmPlan p;
    std::string err;
    if (!plan_einsum(spec, A, B, C, p, err)) {
        c->err = err;
        return DCSD_ERR_INVALID_ARG;
    }
    // batched or very short contractions: FP32 products on the CUDA cores
    if (p.NB != 1 || p.M < 1 || p.N < 1 || p.K < 16)
        return nsplit >= 3 ? einsum64(c, spec, alpha, A, B, beta, C) : einsum32(c, spec, alpha, A, B, beta, C);
    TcEngine* e = c->tc;
    int nseg, pa[6], pb[6];
    split_patterns(nsplit, nseg, pa, pb);
    const long Kp = round_up(p.K, TC_BK);
    const long Kt = nseg * Kp;
    // A long contraction onto few output tiles splits K over the SMs
    // (FP32 partial tiles, summed by a second kernel).  Rough time model:
    // 0.4 us per 64-deep k-step and tile wave plus operand packing at
    // 3 TB/s, against 5 TFLOP/s of the FP32 CUDA-core kernel on its 64 x 64
    // tiles; the faster one runs.
    int ksplit = 1;
    {
        const long nkt = Kt / TC_BK;
        const long bn = p.N >= 256 ? 256 : 128;
        const long tilesMN = ((p.M + TC_BM - 1) / TC_BM) * ((p.N + bn - 1) / bn);
        if (tilesMN <= c->num_sms / 2 && nkt >= 64)
            ksplit = (int)std::max<long>(1, std::min<long>(c->num_sms / tilesMN, nkt / 16));
        // BF16X6, the refinement precision: FP32 partial sums over at most
        // kAccBlocks k-blocks, summed in FP64, when the partials fit (the
        // rounding error of an FP32 sum grows with its length, and the long
        // small-output contractions would otherwise dominate its error)
        if (nsplit >= 3) {
            const long need = (nkt + kAccBlocks - 1) / kAccBlocks;
            if (need >= 4 && need > ksplit && (double)need * (double)p.M * (double)p.N * 4.0 <= kAccWorkspaceBytes)
                ksplit = (int)need;
        }
        const long kper = (nkt + ksplit - 1) / ksplit;
        const long waves = (tilesMN * ksplit + c->num_sms - 1) / std::max(1, c->num_sms);
        const double tc_us = (double)waves * (double)kper * 0.4 + (double)(p.M + p.N) * (double)p.K * 8.0 / 3e6;
        const double simt_us = 2.0 * (double)round_up(p.M, 64) * (double)round_up(p.N, 64) * (double)p.K / 5e6;
        if (simt_us < tc_us)
            return nsplit >= 3 ? einsum64(c, spec, alpha, A, B, beta, C) : einsum32(c, spec, alpha, A, B, beta, C);
    }
    // Row order within M (and N) is free: the packed operand and the
    // epilogue only have to agree.  Order each side's modes by decreasing
    // stride in C, so that its fastest mode is the one closest to C's
    // contiguous axis.
    auto order_modes = [](int nmode, long* size, long* s_op, long* s_c) {
        for (int a = 1; a < nmode; ++a)
            for (int b = a; b > 0 && std::labs(s_c[b - 1]) < std::labs(s_c[b]); --b) {
                std::swap(size[b - 1], size[b]);
                std::swap(s_op[b - 1], s_op[b]);
                std::swap(s_c[b - 1], s_c[b]);
            }
    };
    order_modes(p.nm, p.m_size, p.m_sa, p.m_sc);
    order_modes(p.nn, p.n_size, p.n_sb, p.n_sc);
    // The epilogue maps TMEM lanes (tile rows) to consecutive m: put on the
    // m side the operand whose fastest mode has the smaller stride in C.
    const long m_fast = p.nm > 0 ? std::labs(p.m_sc[p.nm - 1]) : (1l << 62);
    const long n_fast = p.nn > 0 ? std::labs(p.n_sc[p.nn - 1]) : (1l << 62);
    const bool swapped = n_fast < m_fast;
    if (swapped) {
        GemmPlan q = p;
        q.nm = p.nn; q.nn = p.nm; q.M = p.N; q.N = p.M;
        for (int i = 0; i < kMaxMode; ++i) {
            q.m_size[i] = p.n_size[i]; q.m_sa[i] = p.n_sb[i]; q.m_sc[i] = p.n_sc[i];
            q.n_size[i] = p.m_size[i]; q.n_sb[i] = p.m_sa[i]; q.n_sc[i] = p.m_sc[i];
            q.k_sa[i] = p.k_sb[i]; q.k_sb[i] = p.k_sa[i];
        }
        p = q;
    }
    // the m-side operand is the one whose modes p.m_* describe
    const double* msrc = swapped ? B.p : A.p;
    const double* nsrc = swapped ? A.p : B.p;
    const __nv_bfloat16* Apk = nullptr;
    const __nv_bfloat16* Bpk = nullptr;
    DCSD_TRY(pack_operand(c, msrc, p.nm, p.m_size, p.m_sa, p.nk, p.k_size, p.k_sa, p.M, p.K, Kp, nseg, pa,
                          e->pa, Apk));
    DCSD_TRY(pack_operand(c, nsrc, p.nn, p.n_size, p.n_sb, p.nk, p.k_size, p.k_sb, p.N, p.K, Kp, nseg, pb,
                          e->pb, Bpk));
    TcEpi epi;
    std::memset(&epi, 0, sizeof(epi));
    epi.mode = 0;
    epi.C = C.p;
    epi.alpha = alpha;
    epi.beta = beta;
    // accumulation into R2 goes to its FP32 shadow while that is active
    const size_t r2len = 3ul * c->O * c->O * c->V * c->V;
    if (c->r2f_on && beta == 1.0 && C.p >= c->R2 && C.p < c->R2 + r2len) {
        epi.mode = 4;
        epi.C32 = c->r2f + (C.p - c->R2);
    }
    epi.nm = p.nm;
    epi.nn = p.nn;
    for (int i = 0; i < kMaxMode; ++i) {
        epi.m_size[i] = i < p.nm ? p.m_size[i] : 1;
        epi.m_s[i] = i < p.nm ? p.m_sc[i] : 0;
        epi.n_size[i] = i < p.nn ? p.n_size[i] : 1;
        epi.n_s[i] = i < p.nn ? p.n_sc[i] : 0;
    }
    if (ksplit <= 1) return gemm_packed(c, Apk, p.M, Bpk, p.N, Kt, epi);
    // split K: partial tiles, then C (or its FP32 shadow) from their sum
    {
        const int nkt = (int)(Kt / TC_BK), kper = (nkt + ksplit - 1) / ksplit;
        ksplit = (nkt + kper - 1) / kper;
    }
    const size_t wsn = (size_t)ksplit * p.M * p.N;
    if (e->wsk_cap < wsn) {
        if (e->wsk) cudaFree(e->wsk);
        e->wsk = nullptr;
        e->wsk_cap = 0;
        DCSD_CUDA(c, cudaMalloc((void**)&e->wsk, wsn * sizeof(float)));
        e->wsk_cap = wsn;
    }
    TcEpi red = epi;
    red.M = p.M;
    red.N = p.N;
    epi.mode = 5;
    epi.C32 = e->wsk;
    DCSD_TRY(gemm_packed(c, Apk, p.M, Bpk, p.N, Kt, epi, ksplit));
    if (c->trace) trace_begin(c, "tc-splitk-reduce " + c->cur_spec);
    k_tc_splitk_reduce<<<(unsigned)std::max<long>(1, std::min<long>((p.M * p.N + 255) / 256, (long)c->num_sms * 8)),
                         256, 0, c->stream>>>(red, ksplit, e->wsk);
    trace_end(c);
    return launch_check(c, "tc_splitk_reduce");
}

// ---------------------------------------------------------------------------
// particle-particle ladder and its T1 correction on tensor cores
//
//   R2[s][ij][a][b] += sum_cd t_s[ij][cd] (ac|bd)             (s = aa, bb, ab)
//   G[s][ij][k][b]   = sum_cd t_s[ij][cd] (kc|bd)             (s = aa, bb, ab, ab~)
// (ac|bd) = sum_L B_L[a][c] B_L[b][d] is built per chunk of a (resp. k) by a
// tcgen05 GEMM over L whose epilogue writes the tile in BF16 directly in the
// K-major operand layout [(a,b)][(c,d)] of the contraction with the stacked
// amplitudes [(s,i,j)][(c,d)]; the integrals are never stored beyond one
// chunk.  ab~ is the alpha-beta block with (c,d) exchanged.
// ---------------------------------------------------------------------------
// G[s][j][i] = -G[s][i][j] (i < j) and G[s][i][i] = 0 for the same-spin
// blocks s = 0, 1 of G[4][O][O][O][V]
__global__ void k_mirror_pairs(long O, long OV, double* G) {
    const long per = O * O * OV;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < 2 * per; e += (long)gridDim.x * blockDim.x) {
        const long s = e / per, r = e - s * per;
        const long ij = r / OV, kb = r - ij * OV;
        const long i = ij / O, j = ij - i * O;
        if (i < j) continue;
        double* Gs = G + s * per;
        Gs[r] = i == j ? 0.0 : -Gs[(j * O + i) * OV + kb];
    }
}

// Chunks [r0, r0 + nr) of the ladder's first virtual index, nr <= nmax,
// chosen by dynamic programming to minimise the k-steps of the busiest SM
// over the producer and consumer GEMMs of all chunks (each GEMM runs
// ceil(tiles / SMs) waves of tiles of equal work).
static std::vector<std::pair<long, long>> ladder_chunks(long V, long Vp, long rows, long K2t, long Xt, long nmax,
                                                        int sms) {
    auto waves = [&](long M, long N) {
        const long bn = N >= 256 ? 256 : 128;
        const long tiles = ((M + TC_BM - 1) / TC_BM) * ((N + bn - 1) / bn);
        return (tiles + sms - 1) / sms;
    };
    const double launch = 64.0;  // fixed cost of a launch pair, in k-steps
    std::vector<double> best(V + 1, 0.0);
    std::vector<long> pick(V + 1, 1);
    for (long r0 = V - 1; r0 >= 0; --r0) {
        best[r0] = 1e300;
        const long Vb = V - r0;
        // the V tile holds nmax * V rows (r, b); near the end of the triangle
        // (small Vb) more rows r fit, up to the producer A buffer's 4 * nmax
        const long cap = std::min(4 * nmax, std::max(nmax, nmax * V / std::max<long>(1, Vb)));
        for (long nr = 1; nr <= std::min(cap, V - r0); ++nr) {
            const double cost = (double)waves(rows, nr * Vb) * (double)(K2t / TC_BK) +
                                (double)waves(nr * V, Vb * Vp) * (double)(Xt / TC_BK) + launch + best[r0 + nr];
            if (cost < best[r0]) {
                best[r0] = cost;
                pick[r0] = nr;
            }
        }
    }
    std::vector<std::pair<long, long>> out;
    for (long r0 = 0; r0 < V; r0 += pick[r0]) out.push_back({r0, pick[r0]});
    return out;
}

// chunks of a for the symmetric / antisymmetric ladder (dynamic programming
// over the tile waves): per chunk (r0, nr) the producer runs npair x
// #(r, b' >= r) tiles of nkx k-steps (two 128 x 128 MMAs per step, about one
// 128 x 256 step), the consumers GEMMs of rowsM and rowsP rows against
// nr * (V - r0) columns over nks k-steps
static std::vector<std::pair<long, long>> ladder_chunks_sa(long V, long rowsM, long rowsP, long nks, long nkx,
                                                           long npair, long nmax, int sms) {
    auto waves = [&](long M, long N) {
        const long bn = N >= 256 ? 256 : 128;
        const long tiles = ((M + TC_BM - 1) / TC_BM) * ((N + bn - 1) / bn);
        return (tiles + sms - 1) / sms;
    };
    const double launch = 64.0;
    std::vector<double> best(V + 1, 0.0);
    std::vector<long> pick(V + 1, 1);
    for (long r0 = V - 1; r0 >= 0; --r0) {
        best[r0] = 1e300;
        const long Vb = V - r0;
        const long cap = std::min(4 * nmax, std::max(nmax, nmax * V / std::max<long>(1, Vb)));
        for (long nr = 1; nr <= std::min(cap, V - r0); ++nr) {
            const long ptiles = npair * (nr * Vb - nr * (nr - 1) / 2);
            const double cost = (double)((ptiles + sms - 1) / sms) * (double)nkx +
                                (double)(waves(rowsM, nr * Vb) + waves(rowsP, nr * Vb)) * (double)nks + launch +
                                best[r0 + nr];
            if (cost < best[r0]) {
                best[r0] = cost;
                pick[r0] = nr;
            }
        }
    }
    std::vector<std::pair<long, long>> out;
    for (long r0 = 0; r0 < V; r0 += pick[r0]) out.push_back({r0, pick[r0]});
    return out;
}

// R2 += the ladder in symmetric / antisymmetric form (see sa_koff): per chunk
// of a, k_ladder_sa builds the M+ and M- tiles and two consumer GEMMs
// contract them with A- (same-spin pairs and alpha-beta rows) and A+
// (alpha-beta rows), scattering into R2 (codes 0/1/5 and 4 of ladder_scatter).
static dcsd_status ladder_sa_pass(Ctx* c, int nsplit, double* R2, double* G) {
    TcEngine* e = c->tc;
    const long n = c->n, nc = c->nc, O = c->O, V = c->V, X = c->X;
    int nseg, pa[6], pb[6];
    split_patterns(nsplit, nseg, pa, pb);
    const long Vp = round_up(V, 8);
    const long KS = sa_koff(V, Vp), KSp = round_up(KS, TC_BK), KSt = nseg * KSp;
    const long XP = round_up(X, TC_BK), Xt = nseg * XP;
    const int nblk = (int)((Vp + 127) / 128);
    const long YP = (long)nblk * 128;
    const int npair = nblk * (nblk + 1) / 2;
    const long P = O * (O - 1) / 2;
    const long rowsM = 2 * P + O * O, rowsP = O * O;
    if (n * YP >= (1l << 31) || KSt >= (1l << 31) || O >= 1024) {
        c->err = "symmetric / antisymmetric ladder: sizes out of range";
        return DCSD_ERR_INVALID_ARG;
    }
    // consumer row codes: A- rows [same-spin pairs; alpha-beta (block 5)],
    // A+ rows [alpha-beta (block 4)]
    if (e->sa_O != O) {
        std::vector<int> cm(rowsM), cp(rowsP);
        long m = 0;
        for (int sb = 0; sb < 2; ++sb)
            for (long i = 0; i < O; ++i)
                for (long j = i + 1; j < O; ++j) cm[m++] = (sb << 20) | (int)(i << 10) | (int)j;
        for (long i = 0; i < O; ++i)
            for (long j = 0; j < O; ++j) {
                cm[m++] = (5 << 20) | (int)(i << 10) | (int)j;
                cp[i * O + j] = (4 << 20) | (int)(i << 10) | (int)j;
            }
        for (int** pp : {&e->d_code_m, &e->d_code_p})
            if (*pp) { cudaFree(*pp); *pp = nullptr; }
        e->sa_O = -1;
        DCSD_CUDA(c, cudaMalloc((void**)&e->d_code_m, sizeof(int) * rowsM));
        DCSD_CUDA(c, cudaMalloc((void**)&e->d_code_p, sizeof(int) * rowsP));
        DCSD_CUDA(c, cudaMemcpy(e->d_code_m, cm.data(), sizeof(int) * rowsM, cudaMemcpyHostToDevice));
        DCSD_CUDA(c, cudaMemcpy(e->d_code_p, cp.data(), sizeof(int) * rowsP, cudaMemcpyHostToDevice));
        e->sa_O = O;
    }
    // stacked A- and A+ amplitudes (the partial last k-block zeroed first)
    DCSD_TRY(ensure(c, e->sam, (size_t)rowsM * KSt));
    DCSD_TRY(ensure(c, e->sap, (size_t)rowsP * KSt));
    if (KS % TC_BK != 0)
        for (int sg = 0; sg < nseg; ++sg) {
            const long k0 = KS / TC_BK * TC_BK;
            DCSD_CUDA(c, cudaMemsetAsync(e->sam.p + (size_t)sg * rowsM * KSp + (size_t)k0 * rowsM, 0,
                                         sizeof(__nv_bfloat16) * rowsM * TC_BK, c->stream));
            DCSD_CUDA(c, cudaMemsetAsync(e->sap.p + (size_t)sg * rowsP * KSp + (size_t)k0 * rowsP, 0,
                                         sizeof(__nv_bfloat16) * rowsP * TC_BK, c->stream));
        }
    {
        SaPackArgs sp;
        std::memset(&sp, 0, sizeof(sp));
        sp.t2 = c->t2;
        sp.pairoff = e->d_pairoff;
        sp.OO = O * O;
        sp.VV = V * V;
        sp.P2 = (int)(2 * P);
        sp.V = (int)V;
        sp.Vp = (int)Vp;
        sp.ntile = (int)((V + 31) / 32);
        sp.Kp = KSp;
        sp.Am = e->sam.p;
        sp.Ap = e->sap.p;
        sp.rowsM = rowsM;
        sp.rowsP = rowsP;
        sp.nseg = nseg;
        for (int i = 0; i < 6; ++i) sp.pat[i] = pa[i];
        const long work = (2 * P + O * O) * ((long)sp.ntile * (sp.ntile + 1) / 2);
        prof_begin(c, DCSD_PROF_PACK);
        if (c->trace) trace_begin(c, "pack sa-amplitudes rows=" + std::to_string(rowsM + rowsP) + " K=" + std::to_string(KS));
        k_pack_sa<<<(unsigned)std::max<long>(1, std::min<long>(work, (long)c->num_sms * 8)), 256, 0, c->stream>>>(sp);
        trace_end(c);
        prof_end(c, DCSD_PROF_PACK);
        DCSD_TRY(launch_check(c, "pack_sa"));
    }
    // the DF factors B[L][x][nc + y] as [(x, y)][L] for every orbital x (the
    // virtual rows serve the ladder, the occupied ones the G pass), y padded
    // to YP, with the A- and B-side split patterns (B never changes: packed
    // once per split)
    const long xrows = n * YP;
    DCSD_TRY(ensure(c, e->sxa, (size_t)xrows * Xt));
    DCSD_TRY(ensure(c, e->sxb, (size_t)xrows * Xt));
    if (e->sx_nsplit != nsplit) {
        e->sx_nsplit = 0;
        long rsz[2] = {n, YP}, rs[2] = {n, 1};
        long ksz[1] = {X}, ks[1] = {n * n};
        DCSD_TRY(pack(c, c->B + nc, 2, rsz, rs, 1, ksz, ks, xrows, X, XP, nseg, pa, e->sxa.p, V, 1l << 62, nullptr,
                      0, xrows * XP, xrows * 64));
        DCSD_TRY(pack(c, c->B + nc, 2, rsz, rs, 1, ksz, ks, xrows, X, XP, nseg, pb, e->sxb.p, V, 1l << 62, nullptr,
                      0, xrows * XP, xrows * 64));
        e->sx_nsplit = nsplit;
    }
    // M+ and M- tiles of a chunk (zeroed when allocated: rows b' < r and the
    // k padding are never written, and must be finite).  Chunks of up to 16
    // rows a (32 measured slower: the chunk's a rows no longer stay in L2)
    const long chunk = std::max<long>(1, std::min<long>(V, 16));
    for (Buf* b : {&e->svp, &e->svm}) {
        const __nv_bfloat16* old = b->p;
        DCSD_TRY(ensure(c, *b, (size_t)chunk * V * KSt));
        if (b->p != old) DCSD_CUDA(c, cudaMemsetAsync(b->p, 0, b->cap * sizeof(__nv_bfloat16), c->stream));
    }
    const size_t smem = SA_STAGES * 4 * (size_t)SA_TILE + 2048;
    if (!e->sa_attr) {
        DCSD_CUDA(c, cudaFuncSetAttribute(k_ladder_sa, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        e->sa_attr = true;
    }
    CUtensorMap ma, mb;
    DCSD_TRY(make_map_kblk(c, &ma, e->sxa.p, xrows, Xt, 128));
    DCSD_TRY(make_map_kblk(c, &mb, e->sxb.p, xrows, Xt, 128));
    // pass 0, the ladder: chunks of a (triangle b >= a), scatter into R2;
    // pass 1, the G intermediate G[s][i][j][k][b] = sum_cd t[ij][cd] (kc|bd)
    // (s = 3: t with (c,d) exchanged): chunks of occupied k against every b,
    // scatter into G (zeroed first)
    DCSD_CUDA(c, cudaMemsetAsync(G, 0, sizeof(double) * 4 * O * O * O * V, c->stream));
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<std::pair<long, long>> chunks;
        if (pass == 0) chunks = ladder_chunks_sa(V, rowsM, rowsP, KSt / TC_BK, Xt / TC_BK, npair, chunk, c->num_sms);
        else
            for (long k0 = 0; k0 < O; k0 += chunk) chunks.push_back({k0, std::min(chunk, O - k0)});
        for (const auto& ck : chunks) {
            const long r0 = ck.first, nr = ck.second;
            const long Vb = pass == 0 ? V - r0 : V, vrows = nr * Vb;
            SaArgs sa;
            std::memset(&sa, 0, sizeof(sa));
            sa.nkt = (int)(Xt / TC_BK);
            sa.nr = (int)nr;
            sa.Vb = (int)Vb;
            sa.nblk = nblk;
            sa.npair = npair;
            sa.rect = pass;
            sa.ntiles = pass == 0 ? (long)npair * (nr * Vb - nr * (nr - 1) / 2) : (long)npair * nr * Vb;
            sa.xa0 = (int)(pass == 0 ? nc + r0 : r0);
            sa.xb0 = (int)(pass == 0 ? nc + r0 : nc);
            sa.YP = (int)YP;
            sa.V = (int)V;
            sa.Vp = (int)Vp;
            sa.kbs = vrows * 64;
            sa.segstride = vrows * KSp;
            sa.nseg = nseg;
            for (int i = 0; i < 6; ++i) sa.pat[i] = pb[i];
            sa.Vplus = e->svp.p;
            sa.Vminus = e->svm.p;
            prof_begin(c, DCSD_PROF_LADDER);
            if (c->trace) {
                const std::string label = std::string(pass == 0 ? "tc-ladder sa-producer" : "tc-ladder sa-g-producer") +
                                          " nr=" + std::to_string(nr) + " Vb=" + std::to_string(Vb) +
                                          " tiles=" + std::to_string(sa.ntiles) + " Kt=" + std::to_string(Xt);
                if (c->trace_seq) fprintf(stderr, "[dcsd tc #%d] %s\n", c->tc_seq, label.c_str());
                trace_begin(c, label);
            }
            ++c->tc_seq;
            k_ladder_sa<<<(unsigned)std::min<long>(sa.ntiles, c->num_sms), kTcThreads, smem, c->stream>>>(ma, mb, sa,
                                                                                                            e->d_err);
            trace_end(c);
            prof_end(c, DCSD_PROF_LADDER);
            DCSD_TRY(launch_check(c, "ladder_sa"));
            // consumers: A- x M- and A+ x M+, one launch per split product
            TcEpi ce;
            std::memset(&ce, 0, sizeof(ce));
            ce.mode = pass == 0 ? 3 : 6;
            ce.alpha = 1.0;
            ce.C = pass == 0 ? R2 : G;
            ce.C32 = (pass == 0 && c->r2f_on && R2 == c->R2) ? c->r2f : nullptr;
            ce.O = O;
            ce.V = V;
            ce.Vb = Vb;
            ce.a0 = r0;
            ce.OO = O * O;
            ce.VV = V * V;
            for (int sp = 0; sp < nseg; ++sp) {
                ce.rowcode = e->d_code_m;
                DCSD_TRY(gemm_packed(c, e->sam.p + (size_t)sp * rowsM * KSp, rowsM,
                                     e->svm.p + (size_t)sp * vrows * KSp, vrows, KSp, ce, 1, 0, true, true));
                ce.rowcode = e->d_code_p;
                DCSD_TRY(gemm_packed(c, e->sap.p + (size_t)sp * rowsP * KSp, rowsP,
                                     e->svp.p + (size_t)sp * vrows * KSp, vrows, KSp, ce, 1, 0, true, true));
            }
        }
    }
    return DCSD_OK;
}

dcsd_status ladder_tc(Ctx* c, int nsplit, double* R2, double* G) {
    TcEngine* e = c->tc;
    const long n = c->n, nc = c->nc, O = c->O, V = c->V, X = c->X;
    int nseg, pa[6], pb[6];
    split_patterns(nsplit, nseg, pa, pb);
    // (c,d) index of the contraction: c*Vp + d, d padded to a multiple of 8 so
    // that the producer can store 16-byte vectors
    const long Vp = round_up(V, 8);
    const long K2 = V * Vp, K2p = round_up(K2, TC_BK), K2t = nseg * K2p;
    const long XP = round_up(X, TC_BK), Xt = nseg * XP;
    // stacked amplitude rows: the same-spin blocks are antisymmetric in (i,j),
    // so only their pairs i < j are contracted
    const long P = O * (O - 1) / 2;
    const long rows4 = 2 * P + 2 * O * O;
    if (O >= 1024) {
        c->err = "ladder row codes hold occupied indices below 1024";
        return DCSD_ERR_INVALID_ARG;
    }
    if (e->tab_O != O || e->tab_V != V) {
        std::vector<long> pairoff(2 * P > 0 ? 2 * P : 1), growoff(rows4);
        std::vector<int> code(rows4);
        long m = 0;
        for (int s = 0; s < 2; ++s)
            for (long i = 0; i < O; ++i)
                for (long j = i + 1; j < O; ++j, ++m) {
                    pairoff[m] = ((long)s * O * O + i * O + j) * V * V;
                    code[m] = (s << 20) | (int)(i << 10) | (int)j;
                    growoff[m] = ((long)s * O * O + i * O + j) * O * V;
                }
        for (int s = 2; s < 4; ++s)
            for (long i = 0; i < O; ++i)
                for (long j = 0; j < O; ++j, ++m) {
                    code[m] = (s << 20) | (int)(i << 10) | (int)j;
                    growoff[m] = ((long)s * O * O + i * O + j) * O * V;
                }
        for (long** pp : {&e->d_pairoff, &e->d_growoff})
            if (*pp) { cudaFree(*pp); *pp = nullptr; }
        if (e->d_rowcode) { cudaFree(e->d_rowcode); e->d_rowcode = nullptr; }
        e->tab_O = e->tab_V = -1;
        DCSD_CUDA(c, cudaMalloc((void**)&e->d_pairoff, sizeof(long) * pairoff.size()));
        DCSD_CUDA(c, cudaMalloc((void**)&e->d_growoff, sizeof(long) * rows4));
        DCSD_CUDA(c, cudaMalloc((void**)&e->d_rowcode, sizeof(int) * rows4));
        DCSD_CUDA(c, cudaMemcpy(e->d_pairoff, pairoff.data(), sizeof(long) * pairoff.size(), cudaMemcpyHostToDevice));
        DCSD_CUDA(c, cudaMemcpy(e->d_growoff, growoff.data(), sizeof(long) * rows4, cudaMemcpyHostToDevice));
        DCSD_CUDA(c, cudaMemcpy(e->d_rowcode, code.data(), sizeof(int) * rows4, cudaMemcpyHostToDevice));
        e->tab_O = O;
        e->tab_V = V;
    }
    if (c->ladder_sa) {
        // symmetric / antisymmetric form: ladder and G pass
        struct PhaseGuardSa {
            Ctx* c;
            ~PhaseGuardSa() { c->ladder_phase = 0; c->cur_spec = ""; }
        } guard_sa{c};
        c->ladder_phase = 1;
        c->cur_spec = "ladder";
        DCSD_TRY(ladder_sa_pass(c, nsplit, R2, G));
        k_mirror_pairs<<<(unsigned)std::max(1, c->num_sms * 8), 256, 0, c->stream>>>(O, O * V, G);
        return launch_check(c, "mirror_pairs");
    }
    // stacked amplitudes [aa pairs; bb pairs; ab; ab~] x (c,d): segment s is
    // the operand at s * rows4 * K2p, stored K-blocked [K2p / 64][rows4][64] so
    // that each TMA box (64 k x a tile of rows) is one contiguous block
    DCSD_TRY(ensure(c, e->pt, (size_t)rows4 * K2t));
    {
        const long ss = rows4 * K2p, kb = rows4 * 64;
        long rs[1] = {V * V};
        long ksz[2] = {V, Vp}, ks[2] = {V, 1};
        if (P > 0)
            DCSD_TRY(pack(c, c->t2, 0, nullptr, nullptr, 2, ksz, ks, 2 * P, K2, K2p, nseg, pa, e->pt.p, 1l << 62, V,
                          e->d_pairoff, 0, ss, kb));
        long rsz2[1] = {O * O};
        DCSD_TRY(pack(c, c->t2 + 2 * O * O * V * V, 1, rsz2, rs, 2, ksz, ks, O * O, K2, K2p, nseg, pa,
                      e->pt.p + (size_t)2 * P * 64, 1l << 62, V, nullptr, 0, ss, kb));
        long ks2[2] = {1, V};  // (c,d) -> t_ab[ij][d][c]
        DCSD_TRY(pack(c, c->t2 + 2 * O * O * V * V, 1, rsz2, rs, 2, ksz, ks2, O * O, K2, K2p, nseg, pa,
                      e->pt.p + (size_t)(2 * P + O * O) * 64, 1l << 62, V, nullptr, 0, ss, kb));
    }
    // B_vv packed as [(b,d)][L], d padded (B never changes: packed once per
    // split)
    DCSD_TRY(ensure(c, e->pbv, (size_t)K2 * Xt));
    if (e->pbv_nsplit != nsplit) {
        e->pbv_nsplit = 0;
        long rsz[2] = {V, Vp}, rs[2] = {n, 1};
        long ksz[1] = {X}, ks[1] = {n * n};
        DCSD_TRY(pack(c, c->B + nc * n + nc, 2, rsz, rs, 1, ksz, ks, K2, X, XP, nseg, pb, e->pbv.p, V));
        e->pbv_nsplit = nsplit;
    }
    const long chunk = std::max<long>(1, std::min<long>(V, 16));
    {
        // the producer never writes the K padding [V * Vp, K2p) of a V tile:
        // a new buffer starts zeroed, so that padding holds zeros or finite
        // values of earlier tiles (it meets the zero padding of the amplitudes)
        const __nv_bfloat16* old = e->pv.p;
        DCSD_TRY(ensure(c, e->pv, (size_t)chunk * V * K2t));
        if (e->pv.p != old)
            DCSD_CUDA(c, cudaMemsetAsync(e->pv.p, 0, e->pv.cap * sizeof(__nv_bfloat16), c->stream));
    }
    DCSD_TRY(ensure(c, e->pa, (size_t)4 * chunk * V * Xt));
    struct PhaseGuard {
        Ctx* c;
        ~PhaseGuard() { c->ladder_phase = 0; c->cur_spec = ""; }
    } guard{c};
    c->ladder_phase = 1;
    c->cur_spec = "ladder";
    // rows first index a (ladder) then k (correction).  The ladder uses
    // (ac|bd) = (bd|ac): per chunk of a only the columns b >= a0 are built
    // and contracted; the (b,a) elements of the alpha-beta block come from the
    // rows with (c,d) exchanged and same-spin blocks are antisymmetric.
    for (int pass = 0; pass < 2; ++pass) {
        const long R = pass == 0 ? V : O;
        std::vector<std::pair<long, long>> chunks;
        if (pass == 0) chunks = ladder_chunks(V, Vp, rows4, K2t, Xt, chunk, c->num_sms);
        else
            for (long r0 = 0; r0 < R; r0 += chunk) chunks.push_back({r0, std::min(chunk, R - r0)});
        for (const auto& ck : chunks) {
            const long r0 = ck.first, nr = ck.second;
            const long b0 = pass == 0 ? r0 : 0;  // first b column built
            const long Vb = V - b0;
            // producer A: rows (r,c) of B_L[row][c] -> [(r,c)][L]
            {
                long rsz[2] = {nr, V}, rs[2] = {n, 1};
                long ksz[1] = {X}, ks[1] = {n * n};
                const double* src = c->B + (pass == 0 ? (nc + r0) * n + nc : r0 * n + nc);
                DCSD_TRY(pack(c, src, 2, rsz, rs, 1, ksz, ks, nr * V, X, XP, nseg, pa, e->pa.p));
            }
            // producer: tile (r,c) x (b,d) -> V_p[(r,b)][(c,d)] (BF16, consumer-B layout,
            // segment-major and K-blocked like the stacked amplitudes)
            const long vrows = nr * Vb;
            TcEpi pe;
            std::memset(&pe, 0, sizeof(pe));
            pe.mode = 2;
            pe.P = e->pv.p;
            pe.alpha = 1.0;
            pe.nseg = nseg;
            pe.segstride = vrows * K2p;
            for (int i = 0; i < 6; ++i) pe.pat[i] = pb[i];
            pe.V = V;
            pe.Vp = Vp;
            pe.rowlen = K2p;
            pe.kbs = vrows * 64;
            pe.Vb = Vb;
            DCSD_TRY(gemm_packed(c, e->pa.p, nr * V, e->pbv.p + (size_t)b0 * Vp * Xt, Vb * Vp, Xt, pe));
            // consumer: rows (s,i,j) x cols (r,b) over (c,d)
            TcEpi ce;
            std::memset(&ce, 0, sizeof(ce));
            ce.mode = 0;
            ce.alpha = 1.0;
            ce.nm = 1;
            ce.nn = 2;
            for (int i = 0; i < kMaxMode; ++i) { ce.m_size[i] = ce.n_size[i] = 1; ce.m_s[i] = ce.n_s[i] = 0; }
            if (pass == 0) {
                ce.mode = 3;
                ce.C = R2;
                ce.C32 = (c->r2f_on && R2 == c->R2) ? c->r2f : nullptr;
                ce.rowcode = e->d_rowcode;
                ce.O = O;
                ce.V = V;
                ce.Vb = Vb;
                ce.a0 = r0;
                ce.OO = O * O;
                ce.VV = V * V;
                // one launch per split product over its two contiguous segments
                // (the scatter epilogue adds)
                for (int sp = 0; sp < nseg; ++sp)
                    DCSD_TRY(gemm_packed(c, e->pt.p + (size_t)sp * rows4 * K2p, rows4,
                                         e->pv.p + (size_t)sp * vrows * K2p, vrows, K2p, ce, 1, 0, true, true));
            } else {
                ce.C = G + r0 * V;       // G[s][i][j][k][b], row (s,i,j) at the table's offset
                ce.mrow = e->d_growoff;
                ce.m_size[0] = rows4; ce.m_s[0] = O * V;
                ce.n_size[0] = nr; ce.n_s[0] = V;
                ce.n_size[1] = V;  ce.n_s[1] = 1;
                for (int sp = 0; sp < nseg; ++sp) {
                    ce.beta = sp == 0 ? 0.0 : 1.0;
                    DCSD_TRY(gemm_packed(c, e->pt.p + (size_t)sp * rows4 * K2p, rows4,
                                         e->pv.p + (size_t)sp * vrows * K2p, vrows, K2p, ce, 1, 0, true, true));
                }
            }
        }
    }
    // the same-spin G rows (j,i) and (i,i)
    k_mirror_pairs<<<(unsigned)std::max(1, c->num_sms * 8), 256, 0, c->stream>>>(O, O * V, G);
    return launch_check(c, "mirror_pairs");
}

}  // namespace dcsd

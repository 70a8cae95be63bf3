// Strided FP64 contraction engine and elementwise kernels.
//
// Every tensor contraction of the residual is expressed as an einsum spec
// over strided views (no explicit transposes): the planner classifies each
// index letter as batch (A,B,C), m (A,C), n (B,C) or k (A,B), merges
// adjacent modes and hands a GemmPlan to a shared-memory tiled FP64 kernel.
// FP64 has no tcgen05 kind, so this path runs on the CUDA cores; it is the
// parity path of the library and the fallback-free reference for the BF16
// tensor-core engine (tc_gemm.cu) that shares the same planner.
#include "common.h"

#include <algorithm>
#include <cstdio>
#include <cstring>

namespace dcsd {

TV view(double* p, std::initializer_list<long> sizes) {
    TV v;
    v.p = p;
    v.rank = (int)sizes.size();
    int k = 0;
    for (long s : sizes) v.size[k++] = s;
    long st = 1;
    for (int i = v.rank - 1; i >= 0; --i) {
        v.stride[i] = st;
        st *= v.size[i];
    }
    return v;
}

TV sub(TV v, int axis, long start, long len) {
    v.p += start * v.stride[axis];
    v.size[axis] = len;
    return v;
}

TV fix(TV v, int axis, long at) {
    TV r;
    r.p = v.p + at * v.stride[axis];
    r.rank = v.rank - 1;
    int k = 0;
    for (int i = 0; i < v.rank; ++i) {
        if (i == axis) continue;
        r.size[k] = v.size[i];
        r.stride[k] = v.stride[i];
        ++k;
    }
    return r;
}

TV perm(TV v, std::initializer_list<int> order) {
    TV r = v;
    int k = 0;
    for (int a : order) {
        r.size[k] = v.size[a];
        r.stride[k] = v.stride[a];
        ++k;
    }
    return r;
}

// ---------------------------------------------------------------------------
// einsum planner
// ---------------------------------------------------------------------------
namespace {
struct Letter {
    char ch;
    long size;
    long sa, sb, sc;
    bool ina, inb, inc;
};

// merge adjacent modes (listed slow -> fast) when contiguous in every operand
template <int NS>
int merge_modes(int nmode, long* size, long* (&strides)[NS]) {
    int w = 0;
    for (int r = 0; r < nmode; ++r) {
        if (size[r] == 1) continue;
        if (w > 0) {
            bool ok = true;
            for (int s = 0; s < NS; ++s)
                if (strides[s][w - 1] != strides[s][r] * size[r]) ok = false;
            if (ok) {
                size[w - 1] *= size[r];
                for (int s = 0; s < NS; ++s) strides[s][w - 1] = strides[s][r];
                continue;
            }
        }
        size[w] = size[r];
        for (int s = 0; s < NS; ++s) strides[s][w] = strides[s][r];
        ++w;
    }
    return w;
}
}  // namespace

bool plan_einsum(const char* spec, const TV& A, const TV& B, const TV& C,
                 GemmPlan& P, std::string& err) {
    std::string s(spec);
    size_t comma = s.find(','), arrow = s.find("->");
    if (comma == std::string::npos || arrow == std::string::npos || arrow < comma) {
        err = "bad einsum spec " + s;
        return false;
    }
    std::string sa = s.substr(0, comma), sb = s.substr(comma + 1, arrow - comma - 1),
                sc = s.substr(arrow + 2);
    if ((int)sa.size() != A.rank || (int)sb.size() != B.rank || (int)sc.size() != C.rank) {
        err = "einsum rank mismatch for " + s;
        return false;
    }
    std::vector<Letter> L;
    auto find = [&](char ch) -> Letter* {
        for (auto& l : L)
            if (l.ch == ch) return &l;
        L.push_back(Letter{ch, -1, 0, 0, 0, false, false, false});
        return &L.back();
    };
    auto add = [&](const std::string& idx, const TV& t, int which) -> bool {
        for (int i = 0; i < (int)idx.size(); ++i) {
            Letter* l = find(idx[i]);
            bool& in = which == 0 ? l->ina : which == 1 ? l->inb : l->inc;
            if (in) {
                err = "repeated index in one operand: " + s;
                return false;
            }
            in = true;
            if (l->size >= 0 && l->size != t.size[i]) {
                err = "size mismatch for index " + std::string(1, idx[i]) + " in " + s;
                return false;
            }
            l->size = t.size[i];
            (which == 0 ? l->sa : which == 1 ? l->sb : l->sc) = t.stride[i];
        }
        return true;
    };
    if (!add(sa, A, 0) || !add(sb, B, 1) || !add(sc, C, 2)) return false;

    long bsz[kMaxRank], bsa[kMaxRank], bsb[kMaxRank], bsc[kMaxRank];
    long msz[kMaxRank], msa[kMaxRank], msc[kMaxRank];
    long nsz[kMaxRank], nsb[kMaxRank], nsc[kMaxRank];
    long ksz[kMaxRank], ksa[kMaxRank], ksb[kMaxRank];
    int nb = 0, nm = 0, nn = 0, nk = 0;
    // batch / m / n in C order; k in A order
    for (char ch : sc) {
        Letter* l = find(ch);
        if (l->ina && l->inb) {
            bsz[nb] = l->size; bsa[nb] = l->sa; bsb[nb] = l->sb; bsc[nb] = l->sc; ++nb;
        } else if (l->ina) {
            msz[nm] = l->size; msa[nm] = l->sa; msc[nm] = l->sc; ++nm;
        } else if (l->inb) {
            nsz[nn] = l->size; nsb[nn] = l->sb; nsc[nn] = l->sc; ++nn;
        } else {
            err = "output index absent from inputs in " + s;
            return false;
        }
    }
    for (char ch : sa) {
        Letter* l = find(ch);
        if (l->inc) continue;
        if (!l->inb) {
            err = "index summed in one operand only: " + s;
            return false;
        }
        ksz[nk] = l->size; ksa[nk] = l->sa; ksb[nk] = l->sb; ++nk;
    }
    for (char ch : sb) {
        Letter* l = find(ch);
        if (!l->ina && !l->inc) {
            err = "index summed in one operand only: " + s;
            return false;
        }
    }
    {
        long* st[3] = {bsa, bsb, bsc};
        nb = merge_modes<3>(nb, bsz, st);
    }
    {
        long* st[2] = {msa, msc};
        nm = merge_modes<2>(nm, msz, st);
    }
    {
        long* st[2] = {nsb, nsc};
        nn = merge_modes<2>(nn, nsz, st);
    }
    {
        long* st[2] = {ksa, ksb};
        nk = merge_modes<2>(nk, ksz, st);
    }
    if (nb > kMaxMode || nm > kMaxMode || nn > kMaxMode || nk > kMaxMode) {
        err = "too many unmergeable modes in " + s;
        return false;
    }
    P = GemmPlan();
    P.nb = nb; P.nm = nm; P.nn = nn; P.nk = nk;
    P.NB = P.M = P.N = P.K = 1;
    for (int i = 0; i < nb; ++i) {
        P.b_size[i] = bsz[i]; P.b_sa[i] = bsa[i]; P.b_sb[i] = bsb[i]; P.b_sc[i] = bsc[i];
        P.NB *= bsz[i];
    }
    for (int i = 0; i < nm; ++i) {
        P.m_size[i] = msz[i]; P.m_sa[i] = msa[i]; P.m_sc[i] = msc[i];
        P.M *= msz[i];
    }
    for (int i = 0; i < nn; ++i) {
        P.n_size[i] = nsz[i]; P.n_sb[i] = nsb[i]; P.n_sc[i] = nsc[i];
        P.N *= nsz[i];
    }
    for (int i = 0; i < nk; ++i) {
        P.k_size[i] = ksz[i]; P.k_sa[i] = ksa[i]; P.k_sb[i] = ksb[i];
        P.K *= ksz[i];
    }
    for (auto& l : L)
        if (l.size == 0) {
            P.M = 0;  // empty contraction
        }
    return true;
}

static unsigned grid_for(Ctx* c, long total);

// ---------------------------------------------------------------------------
// FP64 tiled GEMM over a GemmPlan
// ---------------------------------------------------------------------------
struct GemmArgs {
    const double* A;
    const double* B;
    double* C;
    double alpha, beta;
    GemmPlan p;
    int a_kfast, b_kfast;
    int nsplit;        // > 1: blockIdx.z = K split, partial tiles -> ws[split][m][n]
    long kchunk;
    double* ws;
};

// linear index -> two offsets; every decomposed index (m, n, k, batch) is
// below 2^31 (checked on the host), so the divisions are 32-bit
__device__ __forceinline__ void decomp2(long idx, int nmode, const long* size, const long* s1,
                                        const long* s2, long& o1, long& o2) {
    o1 = 0;
    o2 = 0;
    unsigned u = (unsigned)idx;
#pragma unroll
    for (int j = kMaxMode - 1; j >= 0; --j) {
        if (j < nmode) {
            const unsigned sz = (unsigned)size[j];
            const unsigned q = u / sz, r = u - q * sz;
            o1 += (long)r * s1[j];
            o2 += (long)r * s2[j];
            u = q;
        }
    }
}

constexpr int GBM = 64, GBN = 64, GBK = 16;

// FP64 input in the product type (integer-unit conversion for FP32)
template <typename T> __device__ __forceinline__ T cvt_in(double x);
template <> __device__ __forceinline__ double cvt_in<double>(double x) { return x; }
template <> __device__ __forceinline__ float cvt_in<float>(double x) { return f64_to_f32(x); }

// T = double: FP64 products and accumulation.  T = float: FP32 products of
// the FP64 inputs (each loaded element is converted once and reused across
// the 64-wide tile), summed in FP32 over one k-tile of GBK and accumulated in
// FP64 across k-tiles.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_t(GemmArgs g) {
    __shared__ T As[GBK][GBM + 1];
    __shared__ T Bs[GBK][GBN + 1];
    __shared__ long rA[GBM], rC[GBM], cB[GBN], cC[GBN];
    __shared__ long kA[GBK], kB[GBK];
    const GemmPlan& p = g.p;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long m0 = (long)blockIdx.x * GBM, n0 = (long)blockIdx.y * GBN;
    const long nbz = g.nsplit > 1 ? 1 : p.NB;
    const long kb = g.nsplit > 1 ? blockIdx.z * g.kchunk : 0;
    const long ke = g.nsplit > 1 ? min(p.K, kb + g.kchunk) : p.K;
    for (long bz = g.nsplit > 1 ? 0 : blockIdx.z; bz < nbz; bz += gridDim.z) {
        long oA = 0, oB = 0, oC = 0;
        {
            long idx = bz;
            for (int j = p.nb - 1; j >= 0; --j) {
                long q = idx / p.b_size[j], r = idx - q * p.b_size[j];
                oA += r * p.b_sa[j]; oB += r * p.b_sb[j]; oC += r * p.b_sc[j];
                idx = q;
            }
        }
        __syncthreads();
        for (int t = tid; t < GBM; t += 256) {
            long m = m0 + t;
            if (m < p.M) decomp2(m, p.nm, p.m_size, p.m_sa, p.m_sc, rA[t], rC[t]);
            else { rA[t] = -1; rC[t] = -1; }
        }
        for (int t = tid; t < GBN; t += 256) {
            long n = n0 + t;
            if (n < p.N) decomp2(n, p.nn, p.n_size, p.n_sb, p.n_sc, cB[t], cC[t]);
            else { cB[t] = -1; cC[t] = -1; }
        }
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        for (long k0 = kb; k0 < ke; k0 += GBK) {
            __syncthreads();
            if (tid < GBK) {
                long k = k0 + tid;
                if (k < ke) decomp2(k, p.nk, p.k_size, p.k_sa, p.k_sb, kA[tid], kB[tid]);
                else { kA[tid] = -1; kB[tid] = -1; }
            }
            __syncthreads();
            for (int e = tid; e < GBM * GBK; e += 256) {
                int mm, kk;
                if (g.a_kfast) { kk = e % GBK; mm = e / GBK; }
                else { mm = e % GBM; kk = e / GBM; }
                long ra = rA[mm], ka = kA[kk];
                As[kk][mm] = (ra >= 0 && ka >= 0) ? cvt_in<T>(g.A[oA + ra + ka]) : (T)0;
            }
            for (int e = tid; e < GBN * GBK; e += 256) {
                int nn, kk;
                if (g.b_kfast) { kk = e % GBK; nn = e / GBK; }
                else { nn = e % GBN; kk = e / GBN; }
                long cb = cB[nn], kb = kB[kk];
                Bs[kk][nn] = (cb >= 0 && kb >= 0) ? cvt_in<T>(g.B[oB + cb + kb]) : (T)0;
            }
            __syncthreads();
            T part[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) part[i][j] = sizeof(T) == 8 ? (T)acc[i][j] : (T)0;
#pragma unroll
            for (int kk = 0; kk < GBK; ++kk) {
                T a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) part[i][j] = fma(a[i], b[j], part[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] = sizeof(T) == 8 ? (double)part[i][j] : acc[i][j] + (double)part[i][j];
        }
        if (g.nsplit > 1) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const long m = m0 + ty + 16 * i;
                if (m >= p.M) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long nn = n0 + tx + 16 * j;
                    if (nn < p.N) g.ws[((long)blockIdx.z * p.M + m) * p.N + nn] = acc[i][j];
                }
            }
            continue;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            long rc = rC[ty + 16 * i];
            if (rc < 0) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                long cc = cC[tx + 16 * j];
                if (cc < 0) continue;
                double* cp = g.C + oC + rc + cc;
                double v = g.alpha * acc[i][j];
                if (g.beta != 0.0) v += g.beta * (*cp);
                *cp = v;
            }
        }
    }
}

// ordered reduction of split-K partials: C = alpha * sum_s ws[s] + beta * C
__global__ void k_splitk_reduce(GemmPlan p, int nsplit, const double* ws, double* C, double alpha,
                                double beta) {
    const long total = p.M * p.N;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
         e += (long)gridDim.x * blockDim.x) {
        const long m = e / p.N, n = e - m * p.N;
        double s = 0.0;
        for (int k = 0; k < nsplit; ++k) s += ws[(long)k * total + e];
        long ra, rc, cb, cc;
        decomp2(m, p.nm, p.m_size, p.m_sa, p.m_sc, ra, rc);
        decomp2(n, p.nn, p.n_size, p.n_sb, p.n_sc, cb, cc);
        double* cp = C + rc + cc;
        double v = alpha * s;
        if (beta != 0.0) v += beta * (*cp);
        *cp = v;
    }
}

// matrix-vector shaped contractions (one output side of extent 1): one warp
// per output element, lanes stride over k
__global__ void __launch_bounds__(256) k_gemv64(GemmArgs g, int vec_is_b) {
    const GemmPlan& p = g.p;
    const long P = vec_is_b ? p.M : p.N;
    const int lane = threadIdx.x & 31;
    for (long o = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5; o < P;
         o += ((long)gridDim.x * blockDim.x) >> 5) {
        long oa, oc, ob = 0;
        if (vec_is_b) decomp2(o, p.nm, p.m_size, p.m_sa, p.m_sc, oa, oc);
        else { decomp2(o, p.nn, p.n_size, p.n_sb, p.n_sc, ob, oc); oa = 0; }
        // four independent partial sums (k, k + 32, k + 64, k + 96), so that
        // the loads of four elements are in flight at once
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        long k = lane;
        for (; k + 96 < p.K; k += 128) {
            long ka0, kb0, ka1, kb1, ka2, kb2, ka3, kb3;
            decomp2(k, p.nk, p.k_size, p.k_sa, p.k_sb, ka0, kb0);
            decomp2(k + 32, p.nk, p.k_size, p.k_sa, p.k_sb, ka1, kb1);
            decomp2(k + 64, p.nk, p.k_size, p.k_sa, p.k_sb, ka2, kb2);
            decomp2(k + 96, p.nk, p.k_size, p.k_sa, p.k_sb, ka3, kb3);
            const double a0 = g.A[oa + ka0], a1 = g.A[oa + ka1], a2 = g.A[oa + ka2], a3 = g.A[oa + ka3];
            const double b0 = g.B[ob + kb0], b1 = g.B[ob + kb1], b2 = g.B[ob + kb2], b3 = g.B[ob + kb3];
            s0 = fma(a0, b0, s0);
            s1 = fma(a1, b1, s1);
            s2 = fma(a2, b2, s2);
            s3 = fma(a3, b3, s3);
        }
        for (; k < p.K; k += 32) {
            long ka, kb;
            decomp2(k, p.nk, p.k_size, p.k_sa, p.k_sb, ka, kb);
            s0 = fma(g.A[oa + ka], g.B[ob + kb], s0);
        }
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
        if (lane == 0) {
            double* cp = g.C + oc;
            double v = g.alpha * s;
            if (g.beta != 0.0) v += g.beta * (*cp);
            *cp = v;
        }
    }
}

static dcsd_status einsum_simt(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B,
                               double beta, const TV& C, bool fp32);

dcsd_status einsum64(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B,
                     double beta, const TV& C) {
    return einsum_simt(c, spec, alpha, A, B, beta, C, false);
}

dcsd_status einsum32(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B,
                     double beta, const TV& C) {
    return einsum_simt(c, spec, alpha, A, B, beta, C, true);
}

void record_einsum(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B, double beta, const TV& C,
                   int engine, int nsplit) {
    TapeOp op;
    op.type = OP_EINSUM;
    op.iarg[1] = engine;  // engine of the adjoint contractions
    op.iarg[2] = nsplit;
    op.spec = spec;
    op.alpha = alpha;
    op.beta = beta;
    op.A = A;
    op.B = B;
    op.C = C;
    rec_push(c, std::move(op));
}

static dcsd_status einsum_simt(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B,
                               double beta, const TV& C, bool fp32) {
    if (c->rec) record_einsum(c, spec, alpha, A, B, beta, C, fp32 ? 1 : 0, 0);
    GemmArgs g;
    std::string err;
    if (!plan_einsum(spec, A, B, C, g.p, err)) {
        c->err = err;
        return DCSD_ERR_INVALID_ARG;
    }
    if (g.p.M == 0 || g.p.N == 0 || g.p.NB == 0) return DCSD_OK;
    if (g.p.M >= (1l << 31) || g.p.N >= (1l << 31) || g.p.K >= (1l << 31) || g.p.NB >= (1l << 31)) {
        c->err = std::string(spec) + ": contraction extent beyond 2^31";
        return DCSD_ERR_INVALID_ARG;
    }
    g.A = A.p;
    g.B = B.p;
    g.C = C.p;
    g.alpha = alpha;
    g.beta = beta;
    g.a_kfast = (g.p.nk > 0 && g.p.k_sa[g.p.nk - 1] == 1) ? 1 : 0;
    g.b_kfast = (g.p.nk > 0 && g.p.k_sb[g.p.nk - 1] == 1) ? 1 : 0;
    g.nsplit = 1;
    g.kchunk = g.p.K;
    g.ws = nullptr;
    if (g.p.NB == 1 && (g.p.N == 1 || g.p.M == 1) && g.p.K >= 64) {
        const int vec_is_b = g.p.N == 1 ? 1 : 0;
        const long outs = vec_is_b ? g.p.M : g.p.N;
        prof_begin(c, DCSD_PROF_FP64);
        if (c->trace)
            trace_begin(c, std::string("fp64-gemv ") + spec + " M=" + std::to_string(g.p.M) + " N=" +
                               std::to_string(g.p.N) + " K=" + std::to_string(g.p.K));
        k_gemv64<<<grid_for(c, outs * 32), 256, 0, c->stream>>>(g, vec_is_b);
        trace_end(c);
        prof_end(c, DCSD_PROF_FP64);
        return launch_check(c, spec);
    }
    const long tiles = ((g.p.M + GBM - 1) / GBM) * ((g.p.N + GBN - 1) / GBN);
    if (g.p.NB == 1 && tiles < c->num_sms && g.p.K >= 2048 && c->splitk_ws) {
        // few output tiles and a long contraction: split K over CTAs
        // about 8 blocks of 256 threads per SM: enough loads in flight to
        // stream the long operands
        long ns = std::min<long>((8 * c->num_sms + tiles - 1) / tiles, g.p.K / 256);
        ns = std::min<long>(ns, (long)(c->splitk_elems / std::max<long>(1, g.p.M * g.p.N)));
        ns = std::min<long>(ns, 65535);
        if (ns >= 2) {
            g.nsplit = (int)ns;
            g.kchunk = ((g.p.K + ns - 1) / ns + GBK - 1) / GBK * GBK;
            g.nsplit = (int)((g.p.K + g.kchunk - 1) / g.kchunk);
            g.ws = c->splitk_ws;
        }
    }
    dim3 grid((unsigned)((g.p.M + GBM - 1) / GBM), (unsigned)((g.p.N + GBN - 1) / GBN),
              (unsigned)(g.nsplit > 1 ? g.nsplit : std::min<long>(g.p.NB, 65535)));
    prof_begin(c, DCSD_PROF_FP64);
    if (c->trace)
        trace_begin(c, std::string(fp32 ? "fp32 " : "fp64 ") + spec + " M=" + std::to_string(g.p.M) + " N=" +
                           std::to_string(g.p.N) + " K=" + std::to_string(g.p.K) + " B=" +
                           std::to_string(g.p.NB) + " split=" + std::to_string(g.nsplit));
    if (fp32) k_gemm_t<float><<<grid, 256, 0, c->stream>>>(g);
    else k_gemm_t<double><<<grid, 256, 0, c->stream>>>(g);
    if (g.nsplit > 1) {
        long tot = g.p.M * g.p.N;
        k_splitk_reduce<<<grid_for(c, tot), 256, 0, c->stream>>>(g.p, g.nsplit, g.ws, g.C, alpha, beta);
    }
    trace_end(c);
    prof_end(c, DCSD_PROF_FP64);
    return launch_check(c, spec);
}

// ---------------------------------------------------------------------------
// generic strided elementwise helpers (rank <= 6)
// ---------------------------------------------------------------------------
struct EwArgs {
    int rank;
    long size[6];
    long sa[6], sc[6];
    long total;
    const double* A;
    double* C;
    double alpha, beta;
};

// linear index -> (offset in A, offset in C); I = unsigned when the element
// count fits 32 bits (cheaper divisions)
template <typename I>
__device__ __forceinline__ void ew_offsets(const EwArgs& a, I idx, long& oa, long& oc) {
    oa = 0;
    oc = 0;
    for (int j = a.rank - 1; j > 0; --j) {
        const I sz = (I)a.size[j];
        const I q = idx / sz, r = idx - q * sz;
        oa += (long)r * a.sa[j];
        oc += (long)r * a.sc[j];
        idx = q;
    }
    oa += (long)idx * a.sa[0];
    oc += (long)idx * a.sc[0];
}

template <typename I>
__global__ void k_axpy_view(EwArgs a) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < a.total;
         e += (long)gridDim.x * blockDim.x) {
        long oa, oc;
        ew_offsets<I>(a, (I)e, oa, oc);
        double v = a.alpha * a.A[oa];
        if (a.beta != 0.0) v += a.beta * a.C[oc];
        a.C[oc] = v;
    }
}

// Shapes and strides of A and C, with size-1 modes dropped and adjacent
// modes merged where both views are contiguous across them.
static bool ew_setup(Ctx* c, const TV& A, const TV& C, EwArgs& a) {
    if (A.rank != C.rank || A.rank > 6) {
        c->err = "elementwise view rank mismatch";
        return false;
    }
    a.rank = 0;
    a.total = 1;
    for (int i = 0; i < A.rank; ++i) {
        if (A.size[i] != C.size[i]) {
            c->err = "elementwise view size mismatch";
            return false;
        }
        a.total *= A.size[i];
        if (A.size[i] == 1) continue;
        if (a.rank > 0 && a.sa[a.rank - 1] == A.stride[i] * A.size[i] &&
            a.sc[a.rank - 1] == C.stride[i] * A.size[i]) {
            a.size[a.rank - 1] *= A.size[i];
            a.sa[a.rank - 1] = A.stride[i];
            a.sc[a.rank - 1] = C.stride[i];
            continue;
        }
        a.size[a.rank] = A.size[i];
        a.sa[a.rank] = A.stride[i];
        a.sc[a.rank] = C.stride[i];
        ++a.rank;
    }
    if (a.rank == 0) {
        a.rank = 1;
        a.size[0] = 1;
        a.sa[0] = a.sc[0] = 0;
    }
    return true;
}

static unsigned grid_for(Ctx* c, long total) {
    long g = (total + 255) / 256;
    long cap = (long)std::max(c->num_sms, 1) * 16;
    return (unsigned)std::max<long>(1, std::min(g, cap));
}

dcsd_status axpy_view(Ctx* c, double alpha, const TV& A, double beta, const TV& C) {
    if (c->rec) {
        TapeOp op;
        op.type = OP_AXPY;
        op.alpha = alpha;
        op.beta = beta;
        op.A = A;
        op.C = C;
        rec_push(c, std::move(op));
    }
    EwArgs a;
    if (!ew_setup(c, A, C, a)) return DCSD_ERR_INVALID_ARG;
    if (a.total == 0) return DCSD_OK;
    a.A = A.p;
    a.C = C.p;
    a.alpha = alpha;
    a.beta = beta;
    if (c->trace) trace_begin(c, "axpy rank=" + std::to_string(a.rank) + " n=" + std::to_string(a.total));
    if (a.total < (1l << 32)) k_axpy_view<unsigned><<<grid_for(c, a.total), 256, 0, c->stream>>>(a);
    else k_axpy_view<unsigned long><<<grid_for(c, a.total), 256, 0, c->stream>>>(a);
    trace_end(c);
    return launch_check(c, "axpy_view");
}

// C[i0,i1,i2,i3] += sum_k alpha_k * A_k[i0,i1,i2,i3] for up to 4 strided views
// (rank 4); one pass over C.  Rows (i0,i1) per block, (i2,i3) per thread.
struct Axpy4Args {
    int nv;
    long size[4];
    long sc[4];
    long sa[4][4];
    const double* A[4];
    double alpha[4];
    double* C;
};

__global__ void __launch_bounds__(256) k_axpy4(Axpy4Args a) {
    const long nrow = a.size[0] * a.size[1], ncol = a.size[2] * a.size[3];
    for (long row = blockIdx.x; row < nrow; row += gridDim.x) {
        const long i0 = row / a.size[1], i1 = row - i0 * a.size[1];
        long rb[4];
        for (int k = 0; k < 4; ++k) rb[k] = i0 * a.sa[k][0] + i1 * a.sa[k][1];
        const long cb = i0 * a.sc[0] + i1 * a.sc[1];
        for (long e = threadIdx.x; e < ncol; e += blockDim.x) {
            const long i2 = e / a.size[3], i3 = e - i2 * a.size[3];
            double v = a.C[cb + i2 * a.sc[2] + i3 * a.sc[3]];
            for (int k = 0; k < a.nv; ++k) v += a.alpha[k] * a.A[k][rb[k] + i2 * a.sa[k][2] + i3 * a.sa[k][3]];
            a.C[cb + i2 * a.sc[2] + i3 * a.sc[3]] = v;
        }
    }
}

static void record_axpy4(Ctx* c, int nv, const double* alpha, const TV* A, const TV& C) {
    TapeOp op;
    op.type = OP_AXPY4;
    op.nv = std::min(nv, 4);
    for (int k = 0; k < op.nv; ++k) {
        op.X[k] = A[k];
        op.al[k] = alpha[k];
    }
    op.C = C;
    rec_push(c, std::move(op));
}

dcsd_status axpy4(Ctx* c, int nv, const double* alpha, const TV* A, const TV& C) {
    if (c->rec) record_axpy4(c, nv, alpha, A, C);
    Axpy4Args a;
    if (C.rank != 4 || nv < 1 || nv > 4) {
        c->err = "axpy4 needs rank-4 views";
        return DCSD_ERR_INVALID_ARG;
    }
    a.nv = nv;
    for (int d = 0; d < 4; ++d) { a.size[d] = C.size[d]; a.sc[d] = C.stride[d]; }
    for (int k = 0; k < 4; ++k) {
        a.A[k] = k < nv ? A[k].p : C.p;
        a.alpha[k] = k < nv ? alpha[k] : 0.0;
        for (int d = 0; d < 4; ++d) {
            if (k < nv && (A[k].rank != 4 || A[k].size[d] != C.size[d])) {
                c->err = "axpy4 shape mismatch";
                return DCSD_ERR_INVALID_ARG;
            }
            a.sa[k][d] = k < nv ? A[k].stride[d] : 0;
        }
    }
    a.C = C.p;
    const long nrow = C.size[0] * C.size[1];
    if (c->trace) trace_begin(c, "axpy4 n=" + std::to_string(nrow * C.size[2] * C.size[3]));
    k_axpy4<<<(unsigned)std::max<long>(1, std::min<long>(nrow, (long)c->num_sms * 32)), 256, 0, c->stream>>>(a);
    trace_end(c);
    return launch_check(c, "axpy4");
}

// R[i][j][a][b] += X[i][a][j][b] - X[j][a][i][b] - X[i][b][j][a] + X[j][b][i][a]
// for X [O][V][O][V] and R [O][O][V][V], both contiguous.  With
// D_ij[a][b] = X[i][a][j][b] - X[j][a][i][b] the increment is
// D_ij[a][b] - D_ij[b][a], and D_ji = -D_ij, so one work item (a pair i < j
// and a pair of 32-wide (a, b) tiles A <= B) reads the four X tiles once and
// updates R[i][j] and R[j][i] on both tiles; for i = j the increment is zero.
__global__ void __launch_bounds__(256) k_ring_antisym(const double* __restrict__ X, double* __restrict__ R, int O,
                                                      int V) {
    __shared__ double dab[32][33], dba[32][33];
    const int nt = (V + 31) / 32;
    const long ntp = (long)nt * (nt + 1) / 2, npair = (long)O * (O - 1) / 2;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const long OV = (long)O * V, VV = (long)V * V;
    for (long w = blockIdx.x; w < npair * ntp; w += gridDim.x) {
        long pr = w / ntp, tp = w - pr * ntp;
        int i = 0;
        while (pr >= O - 1 - i) {
            pr -= O - 1 - i;
            ++i;
        }
        const int j = i + 1 + (int)pr;
        int ta = 0;
        while (tp >= nt - ta) {
            tp -= nt - ta;
            ++ta;
        }
        const int tb = ta + (int)tp;
        const int a0 = 32 * ta, b0 = 32 * tb;
        const double* Xij = X + (long)i * V * OV + (long)j * V;  // X[i][a][j][b] at a * OV + b
        const double* Xji = X + (long)j * V * OV + (long)i * V;
        for (int r = ty; r < 32; r += 8) {
            const long a = a0 + r, b = b0 + tx;            // dab[r][x] = D[a0 + r][b0 + x]
            dab[r][tx] = (a < V && b < V) ? Xij[a * OV + b] - Xji[a * OV + b] : 0.0;
            const long a2 = b0 + r, b2 = a0 + tx;          // dba[r][x] = D[b0 + r][a0 + x]
            dba[r][tx] = (a2 < V && b2 < V) ? Xij[a2 * OV + b2] - Xji[a2 * OV + b2] : 0.0;
        }
        __syncthreads();
        double* Rij = R + ((long)i * O + j) * VV;
        double* Rji = R + ((long)j * O + i) * VV;
        for (int r = ty; r < 32; r += 8) {
            const long a = a0 + r, b = b0 + tx;
            if (a < V && b < V) {
                const double d = dab[r][tx] - dba[tx][r];
                Rij[a * V + b] += d;
                Rji[a * V + b] -= d;
            }
            const long a2 = b0 + r, b2 = a0 + tx;
            if (ta != tb && a2 < V && b2 < V) {
                const double d = dba[r][tx] - dab[tx][r];
                Rij[a2 * V + b2] += d;
                Rji[a2 * V + b2] -= d;
            }
        }
        __syncthreads();
    }
}

static bool contiguous4(const TV& v) {
    return v.rank == 4 && v.stride[3] == 1 && v.stride[2] == v.size[3] && v.stride[1] == v.size[2] * v.size[3] &&
           v.stride[0] == v.size[1] * v.size[2] * v.size[3];
}

dcsd_status ring_antisym_add(Ctx* c, const TV& X, const TV& R) {
    const TV views[4] = {perm(X, {0, 2, 1, 3}), perm(X, {2, 0, 1, 3}), perm(X, {0, 2, 3, 1}), perm(X, {2, 0, 3, 1})};
    const double al[4] = {1.0, -1.0, -1.0, 1.0};
    const long O = R.size[0], V = R.size[2];
    const bool fits = contiguous4(X) && contiguous4(R) && R.size[1] == O && R.size[3] == V && X.size[0] == O &&
                      X.size[1] == V && X.size[2] == O && X.size[3] == V && O < (1l << 20) && V < (1l << 20);
    if (!fits) return axpy4(c, 4, al, views, R);
    if (c->rec) record_axpy4(c, 4, al, views, R);
    const long nt = (V + 31) / 32, work = O * (O - 1) / 2 * (nt * (nt + 1) / 2);
    if (work == 0) return DCSD_OK;
    if (c->trace) trace_begin(c, "ring_antisym n=" + std::to_string(O * O * V * V));
    k_ring_antisym<<<(unsigned)std::max<long>(1, std::min<long>(work, (long)c->num_sms * 16)), 256, 0, c->stream>>>(
        X.p, R.p, (int)O, (int)V);
    trace_end(c);
    return launch_check(c, "ring_antisym");
}

// R[i][j][a][b] += X[j][b][i][a] for X [O][V][O][V] and R [O][O][V][V], both
// contiguous: 32 x 32 (b, a) tiles read along a and written along b through
// shared memory.  Work items: (i, j) and a pair of tiles.
__global__ void __launch_bounds__(256) k_add_swapped(const double* __restrict__ X, double* __restrict__ R, int O,
                                                     int V) {
    __shared__ double t[32][33];
    const int nt = (V + 31) / 32;
    const long ntt = (long)nt * nt, nw = (long)O * O * ntt;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const long OV = (long)O * V, VV = (long)V * V;
    for (long w = blockIdx.x; w < nw; w += gridDim.x) {
        const long ij = w / ntt, tt = w - ij * ntt;
        const long i = ij / O, j = ij - i * O;
        const int a0 = 32 * (int)(tt / nt), b0 = 32 * (int)(tt % nt);
        const double* Xji = X + j * V * OV + i * V;  // X[j][b][i][a] at b * OV + a
        for (int r = ty; r < 32; r += 8) {
            const long b = b0 + r, a = a0 + tx;
            t[r][tx] = (a < V && b < V) ? Xji[b * OV + a] : 0.0;
        }
        __syncthreads();
        double* Rij = R + (i * O + j) * VV;
        for (int r = ty; r < 32; r += 8) {
            const long a = a0 + r, b = b0 + tx;
            if (a < V && b < V) Rij[a * V + b] += t[tx][r];
        }
        __syncthreads();
    }
}

dcsd_status add_swapped(Ctx* c, const TV& X, const TV& R) {
    const long O = R.size[0], V = R.size[2];
    const bool fits = contiguous4(X) && contiguous4(R) && R.size[1] == O && R.size[3] == V && X.size[0] == O &&
                      X.size[1] == V && X.size[2] == O && X.size[3] == V && O < (1l << 20) && V < (1l << 20);
    if (!fits) return axpy_view(c, 1.0, perm(X, {2, 0, 3, 1}), 1.0, R);
    if (c->rec) {
        TapeOp op;
        op.type = OP_AXPY;
        op.alpha = 1.0;
        op.beta = 1.0;
        op.A = perm(X, {2, 0, 3, 1});
        op.C = R;
        rec_push(c, std::move(op));
    }
    const long nt = (V + 31) / 32, work = O * O * nt * nt;
    if (work == 0) return DCSD_OK;
    if (c->trace) trace_begin(c, "add_swapped n=" + std::to_string(O * O * V * V));
    k_add_swapped<<<(unsigned)std::max<long>(1, std::min<long>(work, (long)c->num_sms * 16)), 256, 0, c->stream>>>(
        X.p, R.p, (int)O, (int)V);
    trace_end(c);
    return launch_check(c, "add_swapped");
}

// dots of one vector with up to 16 others in a single pass (contiguous)
struct MultiDotArgs {
    const double* x;
    const double* y[16];
    int m;
    long n;
    double* partial;  // [m][gridDim.x]
};

template <int MM>
__global__ void __launch_bounds__(256) k_multidot_partial(MultiDotArgs a) {
    __shared__ double sh[8][MM];
    double acc[MM];
#pragma unroll
    for (int k = 0; k < MM; ++k) acc[k] = 0.0;
    const long stride = (long)gridDim.x * blockDim.x;
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    // two elements per thread and pass: 2 (m + 1) independent loads in flight
    for (; e + stride < a.n; e += 2 * stride) {
        const double x0 = a.x[e], x1 = a.x[e + stride];
#pragma unroll
        for (int k = 0; k < MM; ++k)
            if (k < a.m) acc[k] = fma(x1, a.y[k][e + stride], fma(x0, a.y[k][e], acc[k]));
    }
    if (e < a.n) {
        const double x0 = a.x[e];
#pragma unroll
        for (int k = 0; k < MM; ++k)
            if (k < a.m) acc[k] = fma(x0, a.y[k][e], acc[k]);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < MM; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < a.m) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += sh[w][threadIdx.x];
        a.partial[(long)threadIdx.x * gridDim.x + blockIdx.x] = v;
    }
}

__global__ void k_multidot_final(const double* partial, int nblk, int m, double* out) {
    const int k = blockIdx.x;
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < nblk; i += 256) s += partial[(long)k * nblk + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

dcsd_status multidot(Ctx* c, const double* x, const double* const* ys_host, int m, long n, double* out) {
    if (m < 1 || m > 16) {
        c->err = "multidot supports 1..16 vectors";
        return DCSD_ERR_INVALID_ARG;
    }
    MultiDotArgs a;
    a.x = x;
    for (int k = 0; k < 16; ++k) a.y[k] = k < m ? ys_host[k] : x;
    a.m = m;
    a.n = n;
    a.partial = c->red;
    // 8 blocks per SM, partials m * nblk <= kRedDoubles
    const int nblk = std::max(1, std::min(8 * std::max(c->num_sms, 1), kRedDoubles / 16));
    trace_begin(c, "multidot");
    if (m <= 1) k_multidot_partial<1><<<nblk, 256, 0, c->stream>>>(a);
    else if (m <= 2) k_multidot_partial<2><<<nblk, 256, 0, c->stream>>>(a);
    else if (m <= 4) k_multidot_partial<4><<<nblk, 256, 0, c->stream>>>(a);
    else if (m <= 8) k_multidot_partial<8><<<nblk, 256, 0, c->stream>>>(a);
    else k_multidot_partial<16><<<nblk, 256, 0, c->stream>>>(a);
    k_multidot_final<<<m, 256, 0, c->stream>>>(c->red, nblk, m, out);
    trace_end(c);
    return launch_check(c, "multidot");
}

// deterministic two-pass dot product
constexpr int kDotBlocks = 1216;  // 8 blocks of 256 threads on each of 152 SMs

template <typename I>
__global__ void k_dot_partial(EwArgs a, const double* B, double* partial) {
    __shared__ double sh[256];
    double s = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < a.total;
         e += (long)gridDim.x * blockDim.x) {
        long oa, ob;
        ew_offsets<I>(a, (I)e, oa, ob);
        s = fma(a.A[oa], B[ob], s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double* partial, int n, double* out, double accumulate) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (accumulate != 0.0 ? *out : 0.0) + sh[0];
}

dcsd_status dot_view(Ctx* c, const TV& A, const TV& B, double* out, double accumulate) {
    if (c->rec) {
        TapeOp op;
        op.type = OP_DOT;
        op.A = A;
        op.B = B;
        op.beta = accumulate;
        op.p[0] = out;
        rec_push(c, std::move(op));
    }
    EwArgs a;
    if (!ew_setup(c, A, B, a)) return DCSD_ERR_INVALID_ARG;
    a.A = A.p;
    a.C = nullptr;
    if (c->trace) trace_begin(c, "dot n=" + std::to_string(a.total));
    if (a.total < (1l << 32)) k_dot_partial<unsigned><<<kDotBlocks, 256, 0, c->stream>>>(a, B.p, c->red);
    else k_dot_partial<unsigned long><<<kDotBlocks, 256, 0, c->stream>>>(a, B.p, c->red);
    trace_end(c);
    DCSD_TRY(launch_check(c, "dot_partial"));
    k_dot_final<<<1, 256, 0, c->stream>>>(c->red, kDotBlocks, out, accumulate);
    return launch_check(c, "dot_final");
}

__global__ void k_fill(double* p, size_t n, double v) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        p[e] = v;
}

dcsd_status fill(Ctx* c, double* p, size_t n, double val) {
    if (n == 0) return DCSD_OK;
    k_fill<<<grid_for(c, (long)n), 256, 0, c->stream>>>(p, n, val);
    return launch_check(c, "fill");
}

// ---------------------------------------------------------------------------
// ABI <-> union layout
// ---------------------------------------------------------------------------
struct LayoutArgs {
    int nc, o, v, O, V;
    int occ_act[2], vir_act[2];
};

__device__ __forceinline__ int occ_map(const LayoutArgs& L, int s, int I) {
    return I < L.nc ? I : L.occ_act[s];
}
__device__ __forceinline__ int vir_map(const LayoutArgs& L, int s, int A) {
    return A == 0 ? L.vir_act[s] : A + 1;
}

static LayoutArgs layout_args(Ctx* c, int ref) {
    LayoutArgs L;
    L.nc = c->nc; L.o = c->o; L.v = c->v; L.O = c->O; L.V = c->V;
    Frame f = frame_of(c, ref);
    for (int s = 0; s < 2; ++s) { L.occ_act[s] = f.occ_act[s]; L.vir_act[s] = f.vir_act[s]; }
    return L;
}

// Row-wise form of the same maps.  dir = 0: every element of the union
// arrays is written (the ABI element it holds, zero where none); one block
// per union doubles row (blk, i', j'), a final block for the singles.
// dir = 1: every ABI element is gathered from its union position; one block
// per ABI doubles row (blk, i, j), a final block for the singles.  Index
// arithmetic is 32-bit within a row (rows of at most 2^31 elements).
__device__ __forceinline__ int occ_inv(const LayoutArgs& L, int s, int u) {
    return u < L.nc ? u : (u == L.occ_act[s] ? L.nc : -1);
}
__device__ __forceinline__ int vir_inv(const LayoutArgs& L, int s, int u) {
    return u == L.vir_act[s] ? 0 : (u >= 2 ? u - 1 : -1);
}

__global__ void __launch_bounds__(256) k_layout_rows(LayoutArgs L, int dir, double* t1, double* t2, double* a1a,
                                                      double* a1b, double* a2aa, double* a2bb, double* a2ab) {
    const int O = L.O, V = L.V, o = L.o, v = L.v;
    const int nrow = dir == 0 ? 3 * O * O : 3 * o * o;
    for (int row = blockIdx.x; row <= nrow; row += gridDim.x) {
        if (row == nrow) {  // singles
            if (dir == 0) {
                for (int e = threadIdx.x; e < 2 * O * V; e += blockDim.x) {
                    const int s = e / (O * V), r = e - s * O * V, ui = r / V, ua = r - ui * V;
                    const int I = occ_inv(L, s, ui), A = vir_inv(L, s, ua);
                    t1[e] = (I >= 0 && A >= 0) ? (s == 0 ? a1a : a1b)[I * v + A] : 0.0;
                }
            } else {
                for (int e = threadIdx.x; e < 2 * o * v; e += blockDim.x) {
                    const int s = e / (o * v), r = e - s * o * v, I = r / v, A = r - I * v;
                    (s == 0 ? a1a : a1b)[r] = t1[((long)s * O + occ_map(L, s, I)) * V + vir_map(L, s, A)];
                }
            }
            continue;
        }
        if (dir == 0) {
            const int blk = row / (O * O), ui = (row / O) % O, uj = row % O;
            const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
            const int i = occ_inv(L, s1, ui), j = occ_inv(L, s2, uj);
            const bool rowok = i >= 0 && j >= 0;
            double* un = t2 + (long)row * V * V;
            const double* ab = (blk == 0 ? a2aa : blk == 1 ? a2bb : a2ab) + (rowok ? ((long)i * o + j) * v * v : 0);
            for (int ua = 0; ua < V; ++ua) {
                const int a = rowok ? vir_inv(L, s1, ua) : -1;
                double* ur = un + (long)ua * V;
                const double* ar = ab + (long)(a >= 0 ? a : 0) * v;
                for (int ub = threadIdx.x; ub < V; ub += blockDim.x) {
                    const int b = vir_inv(L, s2, ub);
                    ur[ub] = (a >= 0 && b >= 0) ? ar[b] : 0.0;
                }
            }
        } else {
            const int blk = row / (o * o), i = (row / o) % o, j = row % o;
            const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
            const int ui = occ_map(L, s1, i), uj = occ_map(L, s2, j);
            const double* un = t2 + (((long)blk * O + ui) * O + uj) * V * V;
            double* ab = (blk == 0 ? a2aa : blk == 1 ? a2bb : a2ab) + ((long)i * o + j) * v * v;
            for (int a = 0; a < v; ++a) {
                const double* ur = un + (long)vir_map(L, s1, a) * V;
                double* ar = ab + (long)a * v;
                for (int b = threadIdx.x; b < v; b += blockDim.x) ar[b] = ur[vir_map(L, s2, b)];
            }
        }
    }
}

static dcsd_status launch_layout(Ctx* c, int ref, int dir, double* u1, double* u2, double* a0, double* a1,
                                 double* a2, double* a3, double* a4, const char* what) {
    LayoutArgs L = layout_args(c, ref);
    const long rows = dir == 0 ? 3l * c->O * c->O : 3l * c->o * c->o;
    if (rows >= (1l << 30) || (long)c->V * c->V >= (1l << 31)) {
        c->err = "layout: sizes out of range";
        return DCSD_ERR_INVALID_ARG;
    }
    if (c->trace) trace_begin(c, "layout");
    k_layout_rows<<<(unsigned)std::min<long>(rows + 1, (long)c->num_sms * 16), 256, 0, c->stream>>>(
        L, dir, u1, u2, a0, a1, a2, a3, a4);
    trace_end(c);
    return launch_check(c, what);
}

dcsd_status unpack_T(Ctx* c, int ref, const double* T1a, const double* T1b, const double* T2aa,
                     const double* T2bb, const double* T2ab) {
    return launch_layout(c, ref, 0, c->t1, c->t2, (double*)T1a, (double*)T1b, (double*)T2aa, (double*)T2bb,
                         (double*)T2ab, "unpack_T");
}

// dir = 0: ABI -> union (every union element written: the ABI element it
// holds, zero elsewhere); dir = 1: union -> ABI (gather)
dcsd_status layout_union(Ctx* c, int ref, int dir, double* u1, double* u2, double* const* abi) {
    return launch_layout(c, ref, dir, u1, u2, abi[0], abi[1], abi[2], abi[3], abi[4], "layout_union");
}

dcsd_status pack_R(Ctx* c, int ref, double* R1a, double* R1b, double* R2aa, double* R2bb,
                   double* R2ab) {
    return launch_layout(c, ref, 1, c->R1, c->R2, R1a, R1b, R2aa, R2bb, R2ab, "pack_R");
}

dcsd_status pack_T(Ctx* c, int ref, double* T1a, double* T1b, double* T2aa, double* T2bb,
                   double* T2ab) {
    return launch_layout(c, ref, 1, c->t1, c->t2, T1a, T1b, T2aa, T2bb, T2ab, "pack_T");
}

// S = 1 - tau, T = 1 + tau with tau[nc + a][k] = t1[spin][k][a]
__global__ void k_tau_mats(int n, int nc, int O, int V, const double* t1s, double* S, double* T) {
    long total = (long)n * n;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
         e += (long)gridDim.x * blockDim.x) {
        int p = (int)(e / n), q = (int)(e % n);
        double tau = 0.0;
        if (p >= nc && q < O) tau = t1s[(long)q * V + (p - nc)];
        double d = p == q ? 1.0 : 0.0;
        S[e] = d - tau;
        T[e] = d + tau;
    }
}

dcsd_status build_tau_mats(Ctx* c, int spin, double* Smat, double* Tmat) {
    if (c->rec) {
        TapeOp op;
        op.type = OP_TAU;
        op.iarg[0] = spin;
        op.A = view(Smat, {(long)c->n, (long)c->n});
        op.B = view(Tmat, {(long)c->n, (long)c->n});
        rec_push(c, std::move(op));
    }
    k_tau_mats<<<grid_for(c, (long)c->n * c->n), 256, 0, c->stream>>>(
        c->n, c->nc, c->O, c->V, c->t1 + (long)spin * c->O * c->V, Smat, Tmat);
    return launch_check(c, "tau_mats");
}

__global__ void k_finite(const double* p, size_t n, double* flag) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
         e += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(p[e])) *flag = 1.0;
}

dcsd_status check_finite(Ctx* c, const double* p, size_t n, double* flag) {
    k_finite<<<grid_for(c, (long)n), 256, 0, c->stream>>>(p, n, flag);
    return launch_check(c, "check_finite");
}

}  // namespace dcsd

namespace dcsd {
void trace_report(Ctx* c) {
    if (!c->trace || c->trace_ev.empty()) return;
    cudaStreamSynchronize(c->stream);
    struct Agg { double ms = 0; long n = 0; };
    std::vector<std::pair<std::string, Agg>> agg;
    double total = 0;
    for (auto& e : c->trace_ev) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e.second.first, e.second.second);
        total += t;
        auto it = std::find_if(agg.begin(), agg.end(), [&](auto& x) { return x.first == e.first; });
        if (it == agg.end()) { agg.push_back({e.first, Agg()}); it = agg.end() - 1; }
        it->second.ms += t;
        it->second.n++;
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    c->trace_ev.clear();
    std::sort(agg.begin(), agg.end(), [](auto& a, auto& b) { return a.second.ms > b.second.ms; });
    fprintf(stderr, "[dcsd trace] total traced %.3f ms\n", total);
    for (auto& a : agg)
        fprintf(stderr, "[dcsd trace] %10.3f ms %5ld x  %s\n", a.second.ms, a.second.n, a.first.c_str());
}
}  // namespace dcsd

// ---------------------------------------------------------------------------
// host execution of a contraction plan (diagnostic of the planner)
// ---------------------------------------------------------------------------
extern "C" dcsd_status dcsd_einsum_host(const char* spec, double alpha, const double* A, int rank_a,
                                        const long* size_a, const long* stride_a, const double* B, int rank_b,
                                        const long* size_b, const long* stride_b, double beta, double* C,
                                        int rank_c, const long* size_c, const long* stride_c) {
    using namespace dcsd;
    if (!spec || !A || !B || !C) return DCSD_ERR_INVALID_ARG;
    TV t[3];
    const int rank[3] = {rank_a, rank_b, rank_c};
    const long* size[3] = {size_a, size_b, size_c};
    const long* stride[3] = {stride_a, stride_b, stride_c};
    for (int x = 0; x < 3; ++x) {
        if (rank[x] < 0 || rank[x] > kMaxRank || (rank[x] > 0 && (!size[x] || !stride[x])))
            return DCSD_ERR_INVALID_ARG;
        t[x].rank = rank[x];
        for (int i = 0; i < rank[x]; ++i) {
            if (size[x][i] < 0) return DCSD_ERR_INVALID_ARG;
            t[x].size[i] = size[x][i];
            t[x].stride[i] = stride[x][i];
        }
    }
    t[0].p = (double*)A;
    t[1].p = (double*)B;
    t[2].p = C;
    GemmPlan P;
    std::string err;
    if (!plan_einsum(spec, t[0], t[1], t[2], P, err)) return DCSD_ERR_INVALID_ARG;
    // offset of linear index idx over n modes (last mode fastest)
    auto off = [](long idx, int n, const long* sz, const long* s) {
        long o = 0;
        for (int j = n - 1; j >= 0; --j) {
            const long q = idx / sz[j];
            o += (idx - q * sz[j]) * s[j];
            idx = q;
        }
        return o;
    };
    for (long bi = 0; bi < P.NB; ++bi) {
        const long oa = off(bi, P.nb, P.b_size, P.b_sa), ob = off(bi, P.nb, P.b_size, P.b_sb),
                   oc = off(bi, P.nb, P.b_size, P.b_sc);
        for (long m = 0; m < P.M; ++m) {
            const long am = oa + off(m, P.nm, P.m_size, P.m_sa), cm = oc + off(m, P.nm, P.m_size, P.m_sc);
            for (long n = 0; n < P.N; ++n) {
                const long bn = ob + off(n, P.nn, P.n_size, P.n_sb), cn = cm + off(n, P.nn, P.n_size, P.n_sc);
                double acc = 0.0;
                for (long k = 0; k < P.K; ++k)
                    acc += A[am + off(k, P.nk, P.k_size, P.k_sa)] * B[bn + off(k, P.nk, P.k_size, P.k_sb)];
                C[cn] = beta != 0.0 ? beta * C[cn] + alpha * acc : alpha * acc;
            }
        }
    }
    return DCSD_OK;
}

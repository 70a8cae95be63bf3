// Two-determinant coupling layer (arXiv 2401.11935, Section II, Eqs. 3-4).
//
// R1_ia   -= W c_ia
// R2_ijab -= W (c_ijab - A(ij;ab)[t_ia c_jb]),     c_q = <A_q| exp(T_B) |B>,
// and the A->B doubles element is zeroed (text after Eq. 4).  T_B is T_A
// with alpha and beta exchanged.  Each c_q is a cluster-to-CI coefficient of
// a determinant at most four-fold excited w.r.t. Phi_B; it is a sum of
// products of at most four amplitudes whose indices are q's own indices or
// the open orbitals t, u.
//
// At context creation the host derives, for every "class" of q (spin block
// and which of q's indices are the open orbitals), the list of amplitude
// products: it applies the excitation operators to occupation strings to
// find the excitation of Phi^A_q relative to Phi_B and its sign, and expands
// the coefficient of that excitation in exp(T1+T2) by peeling off the
// cluster that contains the first hole.  The device kernels then evaluate
// the tables for every element.  Determinant algebra keeps every
// spin-orbital distinct, so terms with a spin-orbital occurring twice never
// arise (the omission the paper makes after Eq. 4).
//
// Determinant convention: spin-orbital id g = spin * n + spatial (alpha
// string first), |D> = a+_{d1} a+_{d2} ... |vac> with d1 < d2 < ...;
// Phi_B is the canonically ordered determinant, which equals E_{A->B} Phi_A
// and puts the singlet at dE_A + W.
#include "common.h"

#include <algorithm>
#include <cstring>

namespace dcsd {

// One amplitude factor of a coupling term.  arr: 0 T1a, 1 T1b, 2 T2aa,
// 3 T2bb, 4 T2ab, 5..7 the T2 blocks with the two virtual indices exchanged
// (so that the element's b index is always the contiguous one).  Index codes:
// 0..3 the element's i, j, a, b; 4/5 the open orbitals t/u as occupied
// (union occ positions n_c, n_c+1); 6/7 t/u as virtual (union vir 0, 1).
struct MFac {
    int8_t arr;
    int8_t idx[4];
};
struct MTerm {
    int8_t sign;
    int8_t nf;
    MFac f[4];
};
constexpr int kNumClasses = 56;  // 48 doubles classes + 8 singles classes
constexpr int kMaxTerms = 640;

struct MTables {
    std::vector<MTerm> terms;
    int off[kNumClasses];
    int cnt[kNumClasses];
};

// tables of both references, identical for every context (they depend only
// on which of q's indices are open orbitals, not on the sizes)
__constant__ MTerm c_terms[2][kMaxTerms];
__constant__ int c_off[2][kNumClasses];
__constant__ int c_cnt[2][kNumClasses];
static bool g_tables_ready[64] = {};

namespace {

using Det = std::vector<int>;

bool annihilate(Det& d, int p, int& sign) {
    auto it = std::find(d.begin(), d.end(), p);
    if (it == d.end()) return false;
    int k = (int)(it - d.begin());
    if (k & 1) sign = -sign;
    d.erase(it);
    return true;
}

bool create(Det& d, int p, int& sign) {
    if (std::find(d.begin(), d.end(), p) != d.end()) return false;
    int k = 0;
    while (k < (int)d.size() && d[k] < p) ++k;
    if (k & 1) sign = -sign;
    d.insert(d.begin() + k, p);
    return true;
}

// E = a+_{A1}..a+_{Ak} a_{Ik}..a_{I1} applied to det
bool excite(Det d, const std::vector<int>& holes, const std::vector<int>& parts, Det& out,
            int& sign) {
    sign = 1;
    for (int h : holes)
        if (!annihilate(d, h, sign)) return false;
    for (int k = (int)parts.size() - 1; k >= 0; --k)
        if (!create(d, parts[k], sign)) return false;
    out = d;
    return true;
}

struct Tok {
    int gid;   // concrete spin-orbital (representative for free tokens)
    int slot;  // -1 fixed; 0..3 = q index i, j, a, b
};
struct SFac {
    int kind;  // 1 = T1, 2 = T2
    Tok t[4];
};
struct STerm {
    int sign;
    std::vector<SFac> f;
};

// coefficient of E_I^A |Phi> in exp(T1+T2)|Phi>: the cluster holding I[0]
// is a single I0->A[p] (sign (-1)^p) or a double (I0,I[q])->(A[p],A[r]),
// p<r (sign (-1)^(p+r+q)), times the coefficient of the remaining excitation
void expand(const std::vector<Tok>& I, const std::vector<Tok>& A, std::vector<STerm>& out) {
    if (I.empty()) {
        out.push_back(STerm{1, {}});
        return;
    }
    const int k = (int)I.size();
    std::vector<Tok> restI(I.begin() + 1, I.end());
    for (int p = 0; p < k; ++p) {
        std::vector<Tok> restA;
        for (int x = 0; x < k; ++x)
            if (x != p) restA.push_back(A[x]);
        std::vector<STerm> sub;
        expand(restI, restA, sub);
        for (auto& s : sub) {
            SFac f{1, {I[0], A[p], Tok{-1, -1}, Tok{-1, -1}}};
            STerm t{((p & 1) ? -1 : 1) * s.sign, {f}};
            t.f.insert(t.f.end(), s.f.begin(), s.f.end());
            out.push_back(t);
        }
    }
    for (int q = 1; q < k; ++q)
        for (int p = 0; p < k; ++p)
            for (int r = p + 1; r < k; ++r) {
                std::vector<Tok> rI, rA;
                for (int x = 1; x < k; ++x)
                    if (x != q) rI.push_back(I[x]);
                for (int x = 0; x < k; ++x)
                    if (x != p && x != r) rA.push_back(A[x]);
                std::vector<STerm> sub;
                expand(rI, rA, sub);
                int sg = ((p + r + q) & 1) ? -1 : 1;
                for (auto& s : sub) {
                    SFac f{2, {I[0], I[q], A[p], A[r]}};
                    STerm t{sg * s.sign, {f}};
                    t.f.insert(t.f.end(), s.f.begin(), s.f.end());
                    out.push_back(t);
                }
            }
}

}  // namespace

static dcsd_status derive_tables(Ctx* c, int ref, MTables& mt) {
    // representative sizes: enough core and external orbitals for two
    // distinct free indices of one kind plus a second set to check signs
    const int nc = 4, nv = 4, n = nc + 2 + nv;
    const int t = nc, u = nc + 1;
    // spatial active orbitals of this frame: occ[spin], vir[spin]
    const int occ_sp[2] = {ref == 0 ? t : u, ref == 0 ? u : t};
    const int vir_sp[2] = {ref == 0 ? u : t, ref == 0 ? t : u};
    auto det_of = [&](int r) {
        Det d;
        int oa = r == 0 ? t : u, ob = r == 0 ? u : t;
        for (int s = 0; s < 2; ++s) {
            for (int p = 0; p < nc; ++p) d.push_back(s * n + p);
            d.push_back(s * n + (s == 0 ? oa : ob));
        }
        std::sort(d.begin(), d.end());
        return d;
    };
    const Det phi_this = det_of(ref), phi_other = det_of(1 - ref);

    mt.terms.clear();
    for (int k = 0; k < kNumClasses; ++k) { mt.off[k] = 0; mt.cnt[k] = 0; }

    // kinds: occ slots use core reps, vir slots use external-virtual reps
    auto run_class = [&](int cls, int nq, const int* spin, const int* act, const int* isocc) -> dcsd_status {
        // representatives (two sets) for free slots
        int rep[2][4];
        bool have2 = true;
        for (int set = 0; set < 2; ++set) {
            for (int q = 0; q < nq; ++q) {
                if (act[q]) {
                    rep[set][q] = spin[q] * n + (isocc[q] ? occ_sp[spin[q]] : vir_sp[spin[q]]);
                    continue;
                }
                int rank = 0;  // how many earlier free slots share the domain
                for (int p = 0; p < q; ++p)
                    if (!act[p] && isocc[p] == isocc[q] && spin[p] == spin[q]) ++rank;
                int idx = rank + set * (rank + 1);  // set 0: 0,1 ; set 1: 1,3
                if (set == 1) idx = rank + 1 + rank;
                int dom = isocc[q] ? nc : nv;
                if (set == 0 && rank >= dom) return DCSD_OK;  // empty class
                if (idx >= dom) { have2 = false; idx = 0; }
                rep[set][q] = spin[q] * n + (isocc[q] ? idx : nc + 2 + idx);
            }
        }
        std::vector<int> holes, parts;
        for (int q = 0; q < nq; ++q) (isocc[q] ? holes : parts).push_back(rep[0][q]);
        Det D;
        int s1;
        if (!excite(phi_this, holes, parts, D, s1)) return DCSD_OK;
        std::vector<int> I, A;
        for (int g : phi_other)
            if (std::find(D.begin(), D.end(), g) == D.end()) I.push_back(g);
        for (int g : D)
            if (std::find(phi_other.begin(), phi_other.end(), g) == phi_other.end()) A.push_back(g);
        Det D2;
        int s2;
        if (!excite(phi_other, I, A, D2, s2) || D2 != D) {
            c->err = "two-determinant table: excitation algebra failed";
            return DCSD_ERR_INVALID_ARG;
        }
        const int s = s1 * s2;
        auto tok_of = [&](int g) {
            for (int q = 0; q < nq; ++q)
                if (!act[q] && rep[0][q] == g) return Tok{g, q};
            return Tok{g, -1};
        };
        std::vector<Tok> It, At;
        for (int g : I) It.push_back(tok_of(g));
        for (int g : A) At.push_back(tok_of(g));
        // value-independence of the sign: re-derive with the second representatives
        if (have2) {
            std::vector<int> h2, p2;
            for (int q = 0; q < nq; ++q) (isocc[q] ? h2 : p2).push_back(rep[1][q]);
            Det Db;
            int sb1, sb2;
            auto conc = [&](const Tok& x) { return x.slot >= 0 ? rep[1][x.slot] : x.gid; };
            std::vector<int> I2, A2;
            for (auto& x : It) I2.push_back(conc(x));
            for (auto& x : At) A2.push_back(conc(x));
            Det Dc;
            if (!excite(phi_this, h2, p2, Db, sb1) || !excite(phi_other, I2, A2, Dc, sb2) ||
                Db != Dc || sb1 * sb2 != s) {
                c->err = "two-determinant table: class sign depends on index values";
                return DCSD_ERR_INVALID_ARG;
            }
        }
        std::vector<STerm> st;
        expand(It, At, st);
        auto spin_of = [&](const Tok& x) { return x.gid / n; };
        // slot codes: 0..3 the element's own index; 4/5 occupied t/u; 6/7 virtual t/u
        auto code = [&](const Tok& x, bool occ) -> int {
            if (x.slot >= 0) return x.slot;
            const int sp = x.gid % n;
            return (occ ? 4 : 6) + (sp == t ? 0 : 1);
        };
        mt.off[cls] = (int)mt.terms.size();
        for (auto& term : st) {
            MTerm m;
            int sign = s * term.sign;
            m.nf = (int8_t)term.f.size();
            bool ok = true;
            for (int k = 0; k < m.nf; ++k) {
                const SFac& f = term.f[k];
                MFac& g = m.f[k];
                if (f.kind == 1) {
                    if (spin_of(f.t[0]) != spin_of(f.t[1])) { ok = false; break; }
                    g.arr = (int8_t)(1 - spin_of(f.t[0]));  // flip: T_other(sigma) = T_this(1-sigma)
                    g.idx[0] = (int8_t)code(f.t[0], true);
                    g.idx[1] = (int8_t)code(f.t[1], false);
                    g.idx[2] = g.idx[3] = 6;
                } else {
                    int so[2] = {1 - spin_of(f.t[0]), 1 - spin_of(f.t[1])};
                    int sv[2] = {1 - spin_of(f.t[2]), 1 - spin_of(f.t[3])};
                    int no_b = so[0] + so[1], nv_b = sv[0] + sv[1];
                    if (no_b != nv_b) { ok = false; break; }
                    int o0 = code(f.t[0], true), o1 = code(f.t[1], true);
                    int v0 = code(f.t[2], false), v1 = code(f.t[3], false);
                    int arr;
                    if (no_b == 0) { arr = 2; }
                    else if (no_b == 2) { arr = 3; }
                    else {
                        arr = 4;
                        if (so[0] == 1) { std::swap(o0, o1); sign = -sign; }
                        if (sv[0] == 1) { std::swap(v0, v1); sign = -sign; }
                    }
                    // keep the element's b (code 3) in the contiguous slot
                    if (v0 == 3) { std::swap(v0, v1); arr += 3; }
                    g.arr = (int8_t)arr;
                    g.idx[0] = (int8_t)o0; g.idx[1] = (int8_t)o1; g.idx[2] = (int8_t)v0; g.idx[3] = (int8_t)v1;
                }
            }
            m.sign = (int8_t)sign;
            if (ok) mt.terms.push_back(m);
        }
        mt.cnt[cls] = (int)mt.terms.size() - mt.off[cls];
        return DCSD_OK;
    };

    const int blk_s1[3] = {0, 1, 0}, blk_s2[3] = {0, 1, 1};
    for (int blk = 0; blk < 3; ++blk)
        for (int bits = 0; bits < 16; ++bits) {
            int act[4] = {(bits >> 3) & 1, (bits >> 2) & 1, (bits >> 1) & 1, bits & 1};
            int spin[4] = {blk_s1[blk], blk_s2[blk], blk_s1[blk], blk_s2[blk]};
            int isocc[4] = {1, 1, 0, 0};
            if (blk != 2 && ((act[0] && act[1]) || (act[2] && act[3]))) continue;  // repeated
            DCSD_TRY(run_class(blk * 16 + bits, 4, spin, act, isocc));
        }
    for (int s = 0; s < 2; ++s)
        for (int bits = 0; bits < 4; ++bits) {
            int act[2] = {(bits >> 1) & 1, bits & 1};
            int spin[2] = {s, s};
            int isocc[2] = {1, 0};
            DCSD_TRY(run_class(48 + s * 4 + bits, 2, spin, act, isocc));
        }
    return DCSD_OK;
}

dcsd_status mtables_build(Ctx* c) {
    if (c->device >= 0 && c->device < 64 && g_tables_ready[c->device]) return DCSD_OK;
    static MTerm h_terms[2][kMaxTerms];
    static int h_off[2][kNumClasses], h_cnt[2][kNumClasses];
    for (int ref = 0; ref < 2; ++ref) {
        MTables mt;
        DCSD_TRY(derive_tables(c, ref, mt));
        if (mt.terms.size() > (size_t)kMaxTerms) {
            c->err = "two-determinant table larger than its constant-memory slot";
            return DCSD_ERR_INVALID_ARG;
        }
        std::memset(h_terms[ref], 0, sizeof(h_terms[ref]));
        std::copy(mt.terms.begin(), mt.terms.end(), h_terms[ref]);
        std::memcpy(h_off[ref], mt.off, sizeof(mt.off));
        std::memcpy(h_cnt[ref], mt.cnt, sizeof(mt.cnt));
    }
    DCSD_CUDA(c, cudaMemcpyToSymbol(c_terms, h_terms, sizeof(h_terms)));
    DCSD_CUDA(c, cudaMemcpyToSymbol(c_off, h_off, sizeof(h_off)));
    DCSD_CUDA(c, cudaMemcpyToSymbol(c_cnt, h_cnt, sizeof(h_cnt)));
    if (c->device >= 0 && c->device < 64) g_tables_ready[c->device] = true;
    return DCSD_OK;
}

void mtables_free(Ctx* c) { (void)c; }

// ---------------------------------------------------------------------------
// device evaluation
// ---------------------------------------------------------------------------
struct MArgs {
    int O, V, nc, ref;
    int occ_act[2], vir_act[2];
    const double* t1;  // [2][O][V]
    const double* t2;  // [3][O][O][V][V]
    const double* t2s; // [3][O][O][V][V] with the virtual indices exchanged
    double* R1;
    double* R2;
    double* c1;        // [2][O][V]
    const double* W;   // device scalar
};

__device__ __forceinline__ double eval_class(const MArgs& a, int cls, const int q[4]) {
    const long O = a.O, V = a.V, nb = O * O * V * V;
    // code -> union position
    const int pos[8] = {q[0], q[1], q[2], q[3], a.nc, a.nc + 1, 0, 1};
    double sum = 0.0;
    const int o = c_off[a.ref][cls], n = c_cnt[a.ref][cls];
    for (int k = 0; k < n; ++k) {
        const MTerm& m = c_terms[a.ref][o + k];
        double prod = (double)m.sign;
        for (int f = 0; f < m.nf; ++f) {
            const MFac& g = m.f[f];
            const int x0 = pos[g.idx[0]], x1 = pos[g.idx[1]];
            double val;
            if (g.arr < 2) {
                val = a.t1[((long)g.arr * O + x0) * V + x1];
            } else {
                const int x2 = pos[g.idx[2]], x3 = pos[g.idx[3]];
                const double* base = g.arr < 5 ? a.t2 + (g.arr - 2) * nb : a.t2s + (g.arr - 5) * nb;
                val = base[(((long)x0 * O + x1) * V + x2) * V + x3];
            }
            prod *= val;
        }
        sum += prod;
    }
    return sum;
}

__device__ __forceinline__ bool occ_ok(const MArgs& a, int s, int i) {
    return i < a.nc || i == a.occ_act[s];
}
__device__ __forceinline__ bool vir_ok(const MArgs& a, int s, int x) {
    return x >= 2 || x == a.vir_act[s];
}

__global__ void k_mterm_singles(MArgs a) {
    const long total = 2l * a.O * a.V;
    const double W = *a.W;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
         e += (long)gridDim.x * blockDim.x) {
        int s = (int)(e / ((long)a.O * a.V));
        int i = (int)((e / a.V) % a.O), x = (int)(e % a.V);
        double cv = 0.0;
        if (occ_ok(a, s, i) && vir_ok(a, s, x)) {
            int cls = 48 + s * 4 + ((i == a.occ_act[s]) << 1) + (x == a.vir_act[s]);
            int q[4] = {i, x, 0, 0};  // slots of a singles class: i, a
            cv = eval_class(a, cls, q);
            a.R1[e] -= W * cv;
        } else {
            a.R1[e] = 0.0;
        }
        a.c1[e] = cv;
    }
}

__global__ void k_mterm_doubles(MArgs a) {
    const long O = a.O, V = a.V;
    const long nblk = O * O * V * V;
    const long total = 3 * nblk;
    const double W = *a.W;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
         e += (long)gridDim.x * blockDim.x) {
        int blk = (int)(e / nblk);
        long r = e - blk * nblk;
        int b = (int)(r % V);
        r /= V;
        int x = (int)(r % V);
        r /= V;
        int j = (int)(r % O);
        int i = (int)(r / O);
        int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
        bool ok = occ_ok(a, s1, i) && occ_ok(a, s2, j) && vir_ok(a, s1, x) && vir_ok(a, s2, b);
        if (blk != 2 && (i == j || x == b)) ok = false;
        if (!ok) {
            a.R2[e] = 0.0;
            continue;
        }
        bool ai = i == a.occ_act[s1], aj = j == a.occ_act[s2];
        bool aa = x == a.vir_act[s1], ab = b == a.vir_act[s2];
        if (blk == 2 && ai && aj && aa && ab) {  // the A->B element
            a.R2[e] = 0.0;
            continue;
        }
        int cls = blk * 16 + (ai << 3) + (aj << 2) + (aa << 1) + ab;
        int q[4] = {i, j, x, b};
        double c2 = eval_class(a, cls, q);
        const double* t1a = a.t1;
        const double* t1b = a.t1 + O * V;
        const double* c1a = a.c1;
        const double* c1b = a.c1 + O * V;
        double tc;
        if (blk == 2) {
            tc = t1a[i * V + x] * c1b[j * V + b] + t1b[j * V + b] * c1a[i * V + x];
        } else {
            const double* t = blk == 0 ? t1a : t1b;
            const double* cc = blk == 0 ? c1a : c1b;
            tc = t[i * V + x] * cc[j * V + b] - t[j * V + x] * cc[i * V + b] -
                 t[i * V + b] * cc[j * V + x] + t[j * V + b] * cc[i * V + x];
        }
        a.R2[e] -= W * (c2 - tc);
    }
}

// t2s[blk][i][j][b][a] = t2[blk][i][j][a][b] (32x32 tiles through shared memory)
__global__ void k_swap_vir(long nmat, int V, const double* t2, double* t2s) {
    __shared__ double tile[32][33];
    const long tv = (V + 31) / 32;
    for (long t = blockIdx.x; t < nmat * tv * tv; t += gridDim.x) {
        const long mat = t / (tv * tv);
        const int ta = (int)((t / tv) % tv), tb = (int)(t % tv);
        const double* src = t2 + mat * (long)V * V;
        double* dst = t2s + mat * (long)V * V;
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
            const int aa = ta * 32 + e / 32, bb = tb * 32 + e % 32;
            tile[e / 32][e % 32] = (aa < V && bb < V) ? src[(long)aa * V + bb] : 0.0;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
            const int bb = tb * 32 + e / 32, aa = ta * 32 + e % 32;
            if (aa < V && bb < V) dst[(long)bb * V + aa] = tile[e % 32][e / 32];
        }
        __syncthreads();
    }
}

dcsd_status apply_mterms(Ctx* c, int ref) {
    MArgs a;
    a.O = c->O; a.V = c->V; a.nc = c->nc; a.ref = ref;
    Frame f = frame_of(c, ref);
    for (int s = 0; s < 2; ++s) { a.occ_act[s] = f.occ_act[s]; a.vir_act[s] = f.vir_act[s]; }
    a.t1 = c->t1; a.t2 = c->t2; a.t2s = c->t2s; a.R1 = c->R1; a.R2 = c->R2; a.c1 = c->c1;
    a.W = c->scal;
    {
        const long nmat = 3l * c->O * c->O, tv = (c->V + 31) / 32;
        const long blocks = std::min<long>(nmat * tv * tv, (long)std::max(c->num_sms, 1) * 16);
        k_swap_vir<<<(unsigned)std::max<long>(1, blocks), 256, 0, c->stream>>>(nmat, c->V, c->t2, c->t2s);
        DCSD_TRY(launch_check(c, "swap_vir"));
    }
    long n1 = 2l * c->O * c->V;
    k_mterm_singles<<<(unsigned)std::max<long>(1, (n1 + 255) / 256), 256, 0, c->stream>>>(a);
    DCSD_TRY(launch_check(c, "mterm_singles"));
    long n2 = 3l * c->O * c->O * c->V * c->V;
    long g = std::min<long>((n2 + 255) / 256, (long)std::max(c->num_sms, 1) * 32);
    k_mterm_doubles<<<(unsigned)g, 256, 0, c->stream>>>(a);
    return launch_check(c, "mterm_doubles");
}

}  // namespace dcsd

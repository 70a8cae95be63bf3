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
        if (mt.cnt[cls] > 64) {
            c->err = "two-determinant class with more than 64 terms";
            return DCSD_ERR_INVALID_ARG;
        }
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

// Largest number of distinct a-only factors / joint (a,b) factors over the
// doubles classes whose a and b are external virtuals (set by mtables_build).
static int g_max_xfac = 0, g_max_hfac = 0;

// In a class with a and b both external, every term has exactly one factor
// holding a and one holding b (each particle index occurs once in a product
// of cluster amplitudes), so a term is either separable -- f(a) g(b) times
// scalars -- or one factor h(a,b) times scalars.  Check that and count the
// distinct symbolic a-factors and (a,b)-factors per class.
static dcsd_status check_separable(Ctx* c, const MTables& mt) {
    for (int blk = 0; blk < 3; ++blk)
        for (int bits = 0; bits < 16; bits += 4) {
            const int cls = blk * 16 + bits;
            std::vector<MFac> xs, hs;
            auto same = [](const MFac& p, const MFac& q) {
                return p.arr == q.arr && std::memcmp(p.idx, q.idx, 4) == 0;
            };
            for (int k = 0; k < mt.cnt[cls]; ++k) {
                const MTerm& m = mt.terms[mt.off[cls] + k];
                int nx = 0, nb = 0, nh = 0;
                MFac xf{}, hf{};
                for (int f = 0; f < m.nf; ++f) {
                    const MFac& g = m.f[f];
                    const int nslot = g.arr < 2 ? 2 : 4;
                    bool ha = false, hb = false;
                    for (int r = 0; r < nslot; ++r) {
                        ha |= g.idx[r] == 2;
                        hb |= g.idx[r] == 3;
                    }
                    if (ha && hb) { ++nh; hf = g; }
                    else if (ha) { ++nx; xf = g; }
                    else if (hb) ++nb;
                }
                if (nh == 1 && nx == 0 && nb == 0) {
                    if (std::none_of(hs.begin(), hs.end(), [&](const MFac& q) { return same(q, hf); }))
                        hs.push_back(hf);
                } else if (nh == 0 && nx == 1 && nb == 1) {
                    if (std::none_of(xs.begin(), xs.end(), [&](const MFac& q) { return same(q, xf); }))
                        xs.push_back(xf);
                } else {
                    c->err = "two-determinant table: a term is neither separable nor a joint factor";
                    return DCSD_ERR_INVALID_ARG;
                }
            }
            g_max_xfac = std::max(g_max_xfac, (int)xs.size());
            g_max_hfac = std::max(g_max_hfac, (int)hs.size());
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
        DCSD_TRY(check_separable(c, mt));
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

// Doubles: one block per (spin block, i, j).  For the class in which a and
// b are external virtuals (all but 2V-1 of the block's elements) the block
// resolves each term's factors once -- with its own i, j substituted -- into
// (pointer, a-stride, b-stride) descriptors; factors that depend on neither
// a nor b are folded into the term's coefficient.  Elements with a or b an
// open orbital use the generic per-element evaluation.
constexpr int kMaxClassTerms = 64;

struct FacDesc {
    const double* base;
    int sa, sb;
};

__global__ void __launch_bounds__(256) k_mterm_doubles(MArgs a) {
    const long O = a.O, V = a.V;
    const long nb = O * O * V * V;
    const int slot = blockIdx.x;
    const int blk = slot / (int)(O * O), i = (slot / (int)O) % (int)O, j = slot % (int)O;
    const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
    double* Rrow = a.R2 + (long)slot * V * V;
    bool rowok = occ_ok(a, s1, i) && occ_ok(a, s2, j);
    if (blk != 2 && i == j) rowok = false;
    if (!rowok) {
        for (long e = threadIdx.x; e < V * V; e += blockDim.x) Rrow[e] = 0.0;
        return;
    }
    const bool ai = i == a.occ_act[s1], aj = j == a.occ_act[s2];
    const int cls_ff = blk * 16 + (ai << 3) + (aj << 2);
    __shared__ FacDesc fac[kMaxClassTerms][4];
    __shared__ double coefS[kMaxClassTerms];
    __shared__ int nfac[kMaxClassTerms];
    const int toff = c_off[a.ref][cls_ff], nterm = min(c_cnt[a.ref][cls_ff], kMaxClassTerms);
    for (int k = threadIdx.x; k < nterm; k += blockDim.x) {
        const MTerm& m = c_terms[a.ref][toff + k];
        double S = (double)m.sign;
        int nf = 0;
        for (int f = 0; f < m.nf; ++f) {
            const MFac& g = m.f[f];
            const double* base;
            long off = 0;
            int sa = 0, sb = 0;
            const int nslot = g.arr < 2 ? 2 : 4;
            const long strides[4] = {g.arr < 2 ? V : O * V * V, g.arr < 2 ? 1 : V * V, V, 1};
            for (int r = 0; r < nslot; ++r) {
                const int cd = g.idx[r];
                const long st = strides[r];
                if (cd == 2) sa += (int)st;
                else if (cd == 3) sb += (int)st;
                else {
                    const int x = cd == 0 ? i : cd == 1 ? j : cd == 4 ? a.nc : cd == 5 ? a.nc + 1 : cd == 6 ? 0 : 1;
                    off += (long)x * st;
                }
            }
            if (g.arr < 2) base = a.t1 + (long)g.arr * O * V + off;
            else if (g.arr < 5) base = a.t2 + (long)(g.arr - 2) * nb + off;
            else base = a.t2s + (long)(g.arr - 5) * nb + off;
            if (sa == 0 && sb == 0) {
                S *= *base;
            } else {
                fac[k][nf].base = base;
                fac[k][nf].sa = sa;
                fac[k][nf].sb = sb;
                ++nf;
            }
        }
        coefS[k] = S;
        nfac[k] = nf;
    }
    __syncthreads();
    const double W = *a.W;
    const double* t1a = a.t1;
    const double* t1b = a.t1 + O * V;
    const double* c1a = a.c1;
    const double* c1b = a.c1 + O * V;
    for (long e = threadIdx.x; e < V * V; e += blockDim.x) {
        const int x = (int)(e / V), b = (int)(e - (long)x * V);
        const bool okx = vir_ok(a, s1, x), okb = vir_ok(a, s2, b);
        if (!okx || !okb || (blk != 2 && x == b)) {
            Rrow[e] = 0.0;
            continue;
        }
        const bool aa = x == a.vir_act[s1], ab = b == a.vir_act[s2];
        if (blk == 2 && ai && aj && aa && ab) {  // the A->B element
            Rrow[e] = 0.0;
            continue;
        }
        double c2;
        if (x >= 2 && b >= 2) {
            c2 = 0.0;
            for (int k = 0; k < nterm; ++k) {
                double prod = coefS[k];
                const int nf = nfac[k];
                for (int f = 0; f < nf; ++f) prod *= fac[k][f].base[(long)x * fac[k][f].sa + (long)b * fac[k][f].sb];
                c2 += prod;
            }
        } else {
            const int cls = blk * 16 + (ai << 3) + (aj << 2) + (aa << 1) + ab;
            const int q[4] = {i, j, x, b};
            c2 = eval_class(a, cls, q);
        }
        double tc;
        if (blk == 2) {
            tc = t1a[i * V + x] * c1b[j * V + b] + t1b[j * V + b] * c1a[i * V + x];
        } else {
            const double* t = blk == 0 ? t1a : t1b;
            const double* cc = blk == 0 ? c1a : c1b;
            tc = t[i * V + x] * cc[j * V + b] - t[j * V + x] * cc[i * V + b] -
                 t[i * V + b] * cc[j * V + x] + t[j * V + b] * cc[i * V + x];
        }
        Rrow[e] -= W * (c2 - tc);
    }
}

// Doubles, separable form: one block per (spin block, i, j).  In the class
// with a and b external the coefficient is
//   c_ijab = sum_d F_d[a] G_d[b] + sum_m s_m H_m[a][b],
// where F_d runs over the distinct a-only factors, G_d[b] collects, for each
// F_d, the coefficient-weighted b-only factors of its terms, and H_m are the
// distinct joint factors with their summed coefficients.  F and G are built
// once per block in shared memory, so an element costs (#F + #H) products
// instead of one product per term.  T is the arithmetic type of the
// contraction: double for the FP64 residual, float for the tensor-core
// precisions (whose residual error is far above FP32 rounding).
constexpr int kMaxXFac = 16, kMaxHFac = 8;

// FP64 value in the contraction type (integer-unit conversion for FP32)
template <typename T> __device__ __forceinline__ T to_t(double x);
template <> __device__ __forceinline__ double to_t<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_t<float>(double x) { return f64_to_f32(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }

template <typename T>
__global__ void __launch_bounds__(256) k_mterm_doubles_sep(MArgs a, int maxx) {
    extern __shared__ __align__(16) unsigned char mt_smem[];
    const long O = a.O, V = a.V;
    const long nb = O * O * V * V;
    const int slot = blockIdx.x;
    const int blk = slot / (int)(O * O), i = (slot / (int)O) % (int)O, j = slot % (int)O;
    const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
    double* Rrow = a.R2 + (long)slot * V * V;
    bool rowok = occ_ok(a, s1, i) && occ_ok(a, s2, j);
    if (blk != 2 && i == j) rowok = false;
    if (!rowok) {
        for (long e = threadIdx.x; e < V * V; e += blockDim.x) Rrow[e] = 0.0;
        return;
    }
    const bool ai = i == a.occ_act[s1], aj = j == a.occ_act[s2];
    const int cls_ff = blk * 16 + (ai << 3) + (aj << 2);
    __shared__ FacDesc fac[kMaxClassTerms][2];
    __shared__ double coefS[kMaxClassTerms];
    __shared__ signed char grp[kMaxClassTerms];  // a-factor group of a separable term, -1 joint
    __shared__ FacDesc xd[kMaxXFac], hd[kMaxHFac];
    __shared__ double hc[kMaxHFac];
    __shared__ int nx_s, nh_s;
    T* F = (T*)mt_smem;           // [maxx][V]: F_d[a]
    T* G = F + (long)maxx * V;    // [maxx][V]: G_d[b]
    const int toff = c_off[a.ref][cls_ff], nterm = min(c_cnt[a.ref][cls_ff], kMaxClassTerms);
    // (1) resolve each term's factors with this block's i, j; fold the
    //     factors that hold neither a nor b into the coefficient
    for (int k = threadIdx.x; k < nterm; k += blockDim.x) {
        const MTerm& m = c_terms[a.ref][toff + k];
        double S = (double)m.sign;
        int nf = 0;
        for (int f = 0; f < m.nf; ++f) {
            const MFac& g = m.f[f];
            long off = 0;
            int sa = 0, sb = 0;
            const int nslot = g.arr < 2 ? 2 : 4;
            const long strides[4] = {g.arr < 2 ? V : O * V * V, g.arr < 2 ? 1 : V * V, V, 1};
            for (int r = 0; r < nslot; ++r) {
                const int cd = g.idx[r];
                const long st = strides[r];
                if (cd == 2) sa += (int)st;
                else if (cd == 3) sb += (int)st;
                else {
                    const int x = cd == 0 ? i : cd == 1 ? j : cd == 4 ? a.nc : cd == 5 ? a.nc + 1 : cd == 6 ? 0 : 1;
                    off += (long)x * st;
                }
            }
            const double* base = g.arr < 2 ? a.t1 + (long)g.arr * O * V + off
                                 : g.arr < 5 ? a.t2 + (long)(g.arr - 2) * nb + off
                                             : a.t2s + (long)(g.arr - 5) * nb + off;
            if (sa == 0 && sb == 0) {
                S *= *base;
            } else if (nf < 2) {
                // order: the a-holding factor first
                if (sb == 0 && nf == 1) {
                    fac[k][1] = fac[k][0];
                    fac[k][0] = FacDesc{base, sa, sb};
                } else {
                    fac[k][nf] = FacDesc{base, sa, sb};
                }
                ++nf;
            }
        }
        coefS[k] = S;
        grp[k] = (signed char)(nf == 1 ? -1 : 0);
    }
    __syncthreads();
    // (2) group the terms (one thread, fixed order: deterministic sums)
    if (threadIdx.x == 0) {
        int nx = 0, nh = 0;
        for (int k = 0; k < nterm; ++k) {
            if (grp[k] < 0) {
                const FacDesc& h = fac[k][0];
                int m = 0;
                while (m < nh && !(hd[m].base == h.base && hd[m].sa == h.sa && hd[m].sb == h.sb)) ++m;
                if (m == nh) {
                    if (nh == kMaxHFac) { nx = maxx + 1; break; }
                    hd[nh] = h;
                    hc[nh] = 0.0;
                    ++nh;
                }
                hc[m] += coefS[k];
            } else {
                const FacDesc& x = fac[k][0];
                int d = 0;
                while (d < nx && !(xd[d].base == x.base && xd[d].sa == x.sa)) ++d;
                if (d == nx) {
                    if (nx == maxx) { nx = maxx + 1; break; }
                    xd[nx++] = x;
                }
                grp[k] = (signed char)d;
            }
        }
        nx_s = nx;
        nh_s = nh;
    }
    __syncthreads();
    // the host bounds both counts; a table outside them takes the per-term
    // evaluation for every element
    const bool generic = nx_s > maxx;
    const int nx = generic ? 0 : nx_s, nh = generic ? 0 : nh_s;
    // (3) F_d[a] and G_d[b]
    for (int b = threadIdx.x; b < V && !generic; b += blockDim.x) {
        for (int d = 0; d < nx; ++d) {
            F[(long)d * V + b] = to_t<T>(xd[d].base[(long)b * xd[d].sa]);
            G[(long)d * V + b] = (T)0;
        }
        for (int k = 0; k < nterm; ++k)
            if (grp[k] >= 0)
                G[(long)grp[k] * V + b] += to_t<T>(coefS[k] * fac[k][1].base[(long)b * fac[k][1].sb]);
    }
    __syncthreads();
    const double W = *a.W;
    const T Wt = to_t<T>(W);
    const double* t1a = a.t1;
    const double* t1b = a.t1 + O * V;
    const double* c1a = a.c1;
    const double* c1b = a.c1 + O * V;
    const double* tA = blk == 1 ? t1b : t1a;  // spin of a (s1)
    const double* cA = blk == 1 ? c1b : c1a;
    const double* tB = blk == 0 ? t1a : t1b;  // spin of b (s2)
    const double* cB = blk == 0 ? c1a : c1b;
    // b-dependent factors of the antisymmetrised t1 c1 product, in T:
    // cj[b] = c_jb, tj[b] = t_jb, ci[b] = c_ib, ti[b] = t_ib (spin of b)
    T* cj = G + (long)maxx * V;
    T* tj = cj + V;
    T* ci = tj + V;
    T* ti = ci + V;
    __shared__ T hcT[kMaxHFac];
    for (int b = threadIdx.x; b < V; b += blockDim.x) {
        cj[b] = to_t<T>(cB[j * V + b]);
        tj[b] = to_t<T>(tB[j * V + b]);
        ci[b] = to_t<T>(cB[i * V + b]);
        ti[b] = to_t<T>(tB[i * V + b]);
    }
    if (threadIdx.x < nh) hcT[threadIdx.x] = to_t<T>(hc[threadIdx.x]);
    __syncthreads();
    // the element's t1 c1 term (b-independent parts passed in)
    auto tc_of = [&](int b, T tia, T cia, T tja, T cja) -> T {
        if (blk == 2) return tia * cj[b] + tj[b] * cia;
        return tia * cj[b] - tja * ci[b] - ti[b] * cja + tj[b] * cia;
    };
    // (4) elements with a and b external: separable form
    const bool zero_diag = blk != 2;
    for (int x = 2; x < V; ++x) {
        const bool okx = vir_ok(a, s1, x);
        const T tia = to_t<T>(tA[i * V + x]), cia = to_t<T>(cA[i * V + x]);
        const T tja = to_t<T>(tA[j * V + x]), cja = to_t<T>(cA[j * V + x]);
        T fx[kMaxXFac];
#pragma unroll
        for (int d = 0; d < kMaxXFac; ++d) fx[d] = d < nx ? F[(long)d * V + x] : (T)0;
        double* Rx = Rrow + (long)x * V;
        for (int b = 2 + threadIdx.x; b < V; b += blockDim.x) {
            if (!okx || (zero_diag && x == b)) {
                Rx[b] = 0.0;
                continue;
            }
            T c2 = (T)0;
            if (!generic) {
#pragma unroll
                for (int d = 0; d < kMaxXFac; ++d)
                    if (d < nx) c2 += fx[d] * G[(long)d * V + b];
                for (int m = 0; m < nh; ++m)
                    c2 += hcT[m] * to_t<T>(hd[m].base[(long)x * hd[m].sa + (long)b * hd[m].sb]);
                // one update per element: a reduction (no load waited for)
                atomicAdd(Rx + b, -to_f64(Wt * (c2 - tc_of(b, tia, cia, tja, cja))));
            } else {
                const int cls = blk * 16 + (ai << 3) + (aj << 2);
                const int q[4] = {i, j, x, b};
                atomicAdd(Rx + b, -(W * (eval_class(a, cls, q) - to_f64(tc_of(b, tia, cia, tja, cja)))));
            }
        }
    }
    // (5) elements with a or b an open orbital: per-term evaluation
    for (int e2 = threadIdx.x; e2 < 4 * (int)V; e2 += blockDim.x) {
        int x, b;
        if (e2 < 2 * (int)V) { x = e2 / (int)V; b = e2 % (int)V; }          // rows a = 0, 1
        else { const int r = e2 - 2 * (int)V; b = r / (int)V; x = r % (int)V; if (x < 2) continue; }  // columns b = 0, 1
        const long e = (long)x * V + b;
        const bool okx = vir_ok(a, s1, x), okb = vir_ok(a, s2, b);
        if (!okx || !okb || (zero_diag && x == b)) {
            Rrow[e] = 0.0;
            continue;
        }
        const bool aa = x == a.vir_act[s1], ab = b == a.vir_act[s2];
        if (blk == 2 && ai && aj && aa && ab) {  // the A->B element
            Rrow[e] = 0.0;
            continue;
        }
        const T tia = to_t<T>(tA[i * V + x]), cia = to_t<T>(cA[i * V + x]);
        const T tja = to_t<T>(tA[j * V + x]), cja = to_t<T>(cA[j * V + x]);
        const int cls = blk * 16 + (ai << 3) + (aj << 2) + (aa << 1) + ab;
        const int q[4] = {i, j, x, b};
        atomicAdd(Rrow + e, -(W * (eval_class(a, cls, q) - to_f64(tc_of(b, tia, cia, tja, cja)))));
    }
}

// ---------------------------------------------------------------------------
// reverse mode of the coupling terms (FP64).  For an element e with
// cotangent g of its residual, R -= W (c - tc) gives W_bar -= g (c - tc),
// c_bar = -W g and tc_bar = W g; c_bar flows to every factor of every term
// of c (product rule), tc_bar to t1 and c1.  Factors are shared between
// elements, so their adjoints accumulate with atomics.
// ---------------------------------------------------------------------------
struct MAdjPtrs {
    double* t1;   // [2][O][V]
    double* t2;   // [3][O][O][V][V]
    double* t2s;  // [3][O][O][V][V] (virtuals exchanged)
    double* c1;   // [2][O][V]
    double* R1;
    double* R2;
    double* scal;  // scal_bar[0] = W_bar
};

__device__ __forceinline__ void eval_class_adj(const MArgs& a, const MAdjPtrs& d, int cls, const int q[4],
                                               double coef) {
    const long O = a.O, V = a.V, nb = O * O * V * V;
    const int pos[8] = {q[0], q[1], q[2], q[3], a.nc, a.nc + 1, 0, 1};
    const int o = c_off[a.ref][cls], n = c_cnt[a.ref][cls];
    for (int k = 0; k < n; ++k) {
        const MTerm& m = c_terms[a.ref][o + k];
        double val[4];
        double* adr[4];
        for (int f = 0; f < m.nf; ++f) {
            const MFac& g = m.f[f];
            const int x0 = pos[g.idx[0]], x1 = pos[g.idx[1]];
            if (g.arr < 2) {
                const long ix = ((long)g.arr * O + x0) * V + x1;
                val[f] = a.t1[ix];
                adr[f] = d.t1 + ix;
            } else {
                const int x2 = pos[g.idx[2]], x3 = pos[g.idx[3]];
                const long ix = (((long)x0 * O + x1) * V + x2) * V + x3;
                if (g.arr < 5) {
                    val[f] = a.t2[(g.arr - 2) * nb + ix];
                    adr[f] = d.t2 + (g.arr - 2) * nb + ix;
                } else {
                    val[f] = a.t2s[(g.arr - 5) * nb + ix];
                    adr[f] = d.t2s + (g.arr - 5) * nb + ix;
                }
            }
        }
        for (int f = 0; f < m.nf; ++f) {
            double prod = coef * (double)m.sign;
            for (int h = 0; h < m.nf; ++h)
                if (h != f) prod *= val[h];
            if (prod != 0.0) atomicAdd(adr[f], prod);
        }
    }
}

__device__ __forceinline__ void block_add(double v, double* target) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(target, v);
}

__global__ void __launch_bounds__(256) k_mterm_doubles_adj(MArgs a, MAdjPtrs d) {
    const long O = a.O, V = a.V, VV = V * V, total = 3 * O * O * VV;
    const double W = *a.W;
    const double* t1a = a.t1;
    const double* t1b = a.t1 + O * V;
    const double* c1a = a.c1;
    const double* c1b = a.c1 + O * V;
    double wbar = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long slot = e / VV, ab = e - slot * VV;
        const int blk = (int)(slot / (O * O)), i = (int)((slot / O) % O), j = (int)(slot % O);
        const int x = (int)(ab / V), b = (int)(ab % V);
        const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
        bool ok = occ_ok(a, s1, i) && occ_ok(a, s2, j) && vir_ok(a, s1, x) && vir_ok(a, s2, b);
        if (blk != 2 && (i == j || x == b)) ok = false;
        const bool ai = i == a.occ_act[s1], aj = j == a.occ_act[s2];
        const bool aa = x == a.vir_act[s1], abv = b == a.vir_act[s2];
        if (blk == 2 && ai && aj && aa && abv) ok = false;  // the A->B element
        if (!ok) {
            d.R2[e] = 0.0;  // the forward overwrote these elements
            continue;
        }
        const double g = d.R2[e];
        if (g == 0.0) continue;
        const int cls = blk * 16 + (ai << 3) + (aj << 2) + (aa << 1) + abv;
        const int q[4] = {i, j, x, b};
        const double c2 = eval_class(a, cls, q);
        double tc;
        const double* tA = blk == 1 ? t1b : t1a;
        const double* cA = blk == 1 ? c1b : c1a;
        const double* tB = blk == 0 ? t1a : t1b;
        const double* cB = blk == 0 ? c1a : c1b;
        const long sA = blk == 1 ? O * V : 0, sB = blk == 0 ? 0 : O * V;
        const double tb = W * g;  // tc_bar
        if (blk == 2) {
            tc = t1a[i * V + x] * c1b[j * V + b] + t1b[j * V + b] * c1a[i * V + x];
            atomicAdd(d.t1 + i * V + x, tb * c1b[j * V + b]);
            atomicAdd(d.c1 + O * V + j * V + b, tb * t1a[i * V + x]);
            atomicAdd(d.t1 + O * V + j * V + b, tb * c1a[i * V + x]);
            atomicAdd(d.c1 + i * V + x, tb * t1b[j * V + b]);
        } else {
            tc = tA[i * V + x] * cB[j * V + b] - tA[j * V + x] * cB[i * V + b] - tB[i * V + b] * cA[j * V + x] +
                 tB[j * V + b] * cA[i * V + x];
            atomicAdd(d.t1 + sA + i * V + x, tb * cB[j * V + b]);
            atomicAdd(d.c1 + sB + j * V + b, tb * tA[i * V + x]);
            atomicAdd(d.t1 + sA + j * V + x, -tb * cB[i * V + b]);
            atomicAdd(d.c1 + sB + i * V + b, -tb * tA[j * V + x]);
            atomicAdd(d.t1 + sB + i * V + b, -tb * cA[j * V + x]);
            atomicAdd(d.c1 + sA + j * V + x, -tb * tB[i * V + b]);
            atomicAdd(d.t1 + sB + j * V + b, tb * cA[i * V + x]);
            atomicAdd(d.c1 + sA + i * V + x, tb * tB[j * V + b]);
        }
        wbar -= g * (c2 - tc);
        eval_class_adj(a, d, cls, q, -W * g);
    }
    block_add(wbar, d.scal);
}

__global__ void __launch_bounds__(256) k_mterm_singles_adj(MArgs a, MAdjPtrs d) {
    const long total = 2l * a.O * a.V;
    const double W = *a.W;
    double wbar = 0.0;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int s = (int)(e / ((long)a.O * a.V));
        const int i = (int)((e / a.V) % a.O), x = (int)(e % a.V);
        if (!(occ_ok(a, s, i) && vir_ok(a, s, x))) {
            d.R1[e] = 0.0;
            continue;
        }
        const double g = d.R1[e];
        wbar -= g * a.c1[e];
        const double cbar = d.c1[e] - W * g;
        if (cbar == 0.0) continue;
        const int cls = 48 + s * 4 + ((i == a.occ_act[s]) << 1) + (x == a.vir_act[s]);
        const int q[4] = {i, x, 0, 0};
        eval_class_adj(a, d, cls, q, cbar);
    }
    block_add(wbar, d.scal);
}

// t2_bar[blk][i][j][a][b] += t2s_bar[blk][i][j][b][a]
__global__ void k_swap_vir_adj(long nmat, int V, const double* t2sb, double* t2b) {
    const long total = nmat * V * V;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long mat = e / ((long)V * V), r = e - mat * V * V;
        const int x = (int)(r / V), b = (int)(r % V);
        t2b[e] += t2sb[mat * V * V + (long)b * V + x];
    }
}

dcsd_status mterms_adjoint(Ctx* c, int ref, double* t1b, double* t2b, double* t2sb, double* c1b, double* R1b,
                           double* R2b, double* scalb) {
    MArgs a;
    a.O = c->O; a.V = c->V; a.nc = c->nc; a.ref = ref;
    Frame f = frame_of(c, ref);
    for (int s = 0; s < 2; ++s) { a.occ_act[s] = f.occ_act[s]; a.vir_act[s] = f.vir_act[s]; }
    a.t1 = c->t1; a.t2 = c->t2; a.t2s = c->t2s; a.R1 = c->R1; a.R2 = c->R2; a.c1 = c->c1;
    a.W = c->scal;
    MAdjPtrs d{t1b, t2b, t2sb, c1b, R1b, R2b, scalb};
    const unsigned g = (unsigned)std::max(1, c->num_sms * 8);
    // doubles first: they add to c1_bar, which the singles then propagate
    k_mterm_doubles_adj<<<g, 256, 0, c->stream>>>(a, d);
    DCSD_TRY(launch_check(c, "mterm_doubles_adj"));
    k_mterm_singles_adj<<<g, 256, 0, c->stream>>>(a, d);
    return launch_check(c, "mterm_singles_adj");
}

dcsd_status swap_vir_adjoint(Ctx* c, const double* t2sb, double* t2b) {
    k_swap_vir_adj<<<(unsigned)std::max(1, c->num_sms * 8), 256, 0, c->stream>>>(3l * c->O * c->O, c->V, t2sb,
                                                                                t2b);
    return launch_check(c, "swap_vir_adj");
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

dcsd_status apply_mterms(Ctx* c, int ref, bool fp32) {
    if (c->rec) {
        TapeOp sw;
        sw.type = OP_SWAPVIR;
        rec_push(c, std::move(sw));
        TapeOp op;
        op.type = OP_MTERMS;
        op.iarg[0] = ref;
        rec_push(c, std::move(op));
    }
    MArgs a;
    a.O = c->O; a.V = c->V; a.nc = c->nc; a.ref = ref;
    Frame f = frame_of(c, ref);
    for (int s = 0; s < 2; ++s) { a.occ_act[s] = f.occ_act[s]; a.vir_act[s] = f.vir_act[s]; }
    a.t1 = c->t1; a.t2 = c->t2; a.t2s = c->t2s; a.R1 = c->R1; a.R2 = c->R2; a.c1 = c->c1;
    a.W = c->scal;
    {
        const long nmat = 3l * c->O * c->O, tv = (c->V + 31) / 32;
        const long blocks = std::min<long>(nmat * tv * tv, (long)std::max(c->num_sms, 1) * 16);
        trace_begin(c, "swap_vir");
        k_swap_vir<<<(unsigned)std::max<long>(1, blocks), 256, 0, c->stream>>>(nmat, c->V, c->t2, c->t2s);
        trace_end(c);
        DCSD_TRY(launch_check(c, "swap_vir"));
    }
    long n1 = 2l * c->O * c->V;
    k_mterm_singles<<<(unsigned)std::max<long>(1, (n1 + 255) / 256), 256, 0, c->stream>>>(a);
    DCSD_TRY(launch_check(c, "mterm_singles"));
    const int maxx = std::max(g_max_xfac, 1);
    const size_t smem = (2ul * maxx + 4) * c->V * (fp32 ? sizeof(float) : sizeof(double));
    const unsigned grid = (unsigned)(3l * c->O * c->O);
    trace_begin(c, fp32 ? "mterm_doubles_sep32" : "mterm_doubles_sep64");
    if (g_max_xfac > kMaxXFac || g_max_hfac > kMaxHFac || smem > 160 * 1024) {
        k_mterm_doubles<<<grid, 256, 0, c->stream>>>(a);  // per-term form (large V)
    } else if (fp32) {
        DCSD_CUDA(c, cudaFuncSetAttribute(k_mterm_doubles_sep<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        k_mterm_doubles_sep<float><<<grid, 256, smem, c->stream>>>(a, maxx);
    } else {
        DCSD_CUDA(c, cudaFuncSetAttribute(k_mterm_doubles_sep<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        k_mterm_doubles_sep<double><<<grid, 256, smem, c->stream>>>(a, maxx);
    }
    trace_end(c);
    return launch_check(c, "mterm_doubles");
}

// Fixed-reference methods (no coupling terms): the residual positions that
// are not amplitudes of the frame (padding of the union layout, same-spin
// diagonals) and the fixed A->B element are set to zero, the same masking
// that the coupling kernels apply to the 2D residual.
__global__ void k_fr_mask(MArgs a) {
    const long O = a.O, V = a.V, n1 = 2 * O * V, total = n1 + 3 * O * O * V * V;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        bool ok;
        if (e < n1) {
            const int s = (int)(e / (O * V)), i = (int)((e / V) % O), x = (int)(e % V);
            ok = occ_ok(a, s, i) && vir_ok(a, s, x);
            if (!ok) a.R1[e] = 0.0;
            continue;
        }
        const long r = e - n1;
        const int blk = (int)(r / (O * O * V * V));
        const int i = (int)((r / (O * V * V)) % O), j = (int)((r / (V * V)) % O);
        const int x = (int)((r / V) % V), b = (int)(r % V);
        const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
        ok = occ_ok(a, s1, i) && occ_ok(a, s2, j) && vir_ok(a, s1, x) && vir_ok(a, s2, b);
        if (blk != 2 && (i == j || x == b)) ok = false;
        if (blk == 2 && i == a.occ_act[s1] && j == a.occ_act[s2] && x == a.vir_act[s1] && b == a.vir_act[s2])
            ok = false;
        if (!ok) a.R2[r] = 0.0;
    }
}

__global__ void k_set_value(double* p, double v) { *p = v; }

dcsd_status apply_fr_mask(Ctx* c, int ref) {
    MArgs a;
    a.O = c->O; a.V = c->V; a.nc = c->nc; a.ref = ref;
    Frame f = frame_of(c, ref);
    for (int s = 0; s < 2; ++s) { a.occ_act[s] = f.occ_act[s]; a.vir_act[s] = f.vir_act[s]; }
    a.t1 = c->t1; a.t2 = c->t2; a.t2s = c->t2s; a.R1 = c->R1; a.R2 = c->R2; a.c1 = c->c1;
    a.W = c->scal;
    const long total = 2l * c->O * c->V + 3l * c->O * c->O * c->V * c->V;
    const long blocks = std::min<long>((total + 255) / 256, (long)std::max(c->num_sms, 1) * 8);
    k_fr_mask<<<(unsigned)std::max<long>(1, blocks), 256, 0, c->stream>>>(a);
    return launch_check(c, "fr_mask");
}

dcsd_status set_fixed_amplitude(Ctx* c, int ref, double value) {
    const Frame f = frame_of(c, ref);
    const long O = c->O, V = c->V;
    const long e = (((2 * O + f.occ_act[0]) * O + f.occ_act[1]) * V + f.vir_act[0]) * V + f.vir_act[1];
    k_set_value<<<1, 1, 0, c->stream>>>(c->t2 + e, value);
    return launch_check(c, "set_fixed_amplitude");
}

}  // namespace dcsd

// ---------------------------------------------------------------------------
// host evaluation of the coupling coefficients from the derived tables
// ---------------------------------------------------------------------------
extern "C" dcsd_status dcsd_coupling_host(int ref, int n_c, int n_v, const double* T1a, const double* T1b,
                                          const double* T2aa, const double* T2bb, const double* T2ab, double* c1a,
                                          double* c1b, double* c2aa, double* c2bb, double* c2ab) {
    using namespace dcsd;
    if ((ref != 0 && ref != 1) || n_c < 0 || n_v < 1 || n_c > 64 || n_v > 64 || !T1a || !T1b || !T2aa ||
        !T2bb || !T2ab || !c1a || !c1b || !c2aa || !c2bb || !c2ab)
        return DCSD_ERR_INVALID_ARG;
    Ctx tmp;  // carries the sizes and error text only; no device state
    tmp.nc = n_c;
    tmp.nv = n_v;
    MTables mt;
    if (derive_tables(&tmp, ref, mt) != DCSD_OK) return DCSD_ERR_INVALID_ARG;
    const long o = n_c + 1, v = n_v + 1, O = n_c + 2, V = n_v + 2;
    const Frame f = frame_of(&tmp, ref);
    // ABI index -> union position (core i < n_c, the spin's active occupied;
    // the spin's active virtual at a = 0, externals a >= 1 at 2 + a - 1)
    auto occ = [&](int s, long i) { return i < n_c ? i : (long)f.occ_act[s]; };
    auto vir = [&](int s, long a) { return a == 0 ? (long)f.vir_act[s] : a + 1; };
    const long nb = O * O * V * V;
    std::vector<double> t1(2 * O * V, 0.0), t2(3 * nb, 0.0), t2s(3 * nb, 0.0);
    const double* T1[2] = {T1a, T1b};
    const double* T2[3] = {T2aa, T2bb, T2ab};
    for (int s = 0; s < 2; ++s)
        for (long i = 0; i < o; ++i)
            for (long a = 0; a < v; ++a) t1[(s * O + occ(s, i)) * V + vir(s, a)] = T1[s][i * v + a];
    for (int blk = 0; blk < 3; ++blk) {
        const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
        for (long i = 0; i < o; ++i)
            for (long j = 0; j < o; ++j)
                for (long a = 0; a < v; ++a)
                    for (long b = 0; b < v; ++b) {
                        const double x = T2[blk][((i * o + j) * v + a) * v + b];
                        const long I = occ(s1, i), J = occ(s2, j), A = vir(s1, a), B = vir(s2, b);
                        t2[blk * nb + ((I * O + J) * V + A) * V + B] = x;
                        t2s[blk * nb + ((I * O + J) * V + B) * V + A] = x;
                    }
    }
    // one class of q: the sum over its terms of sign x product of factors
    auto eval = [&](int cls, const long q[4]) {
        const long pos[8] = {q[0], q[1], q[2], q[3], n_c, n_c + 1, 0, 1};
        double sum = 0.0;
        for (int k = 0; k < mt.cnt[cls]; ++k) {
            const MTerm& m = mt.terms[mt.off[cls] + k];
            double prod = (double)m.sign;
            for (int g = 0; g < m.nf; ++g) {
                const MFac& fa = m.f[g];
                const long x0 = pos[fa.idx[0]], x1 = pos[fa.idx[1]];
                if (fa.arr < 2) {
                    prod *= t1[(fa.arr * O + x0) * V + x1];
                } else {
                    const long x2 = pos[fa.idx[2]], x3 = pos[fa.idx[3]];
                    const std::vector<double>& src = fa.arr < 5 ? t2 : t2s;
                    prod *= src[(fa.arr < 5 ? fa.arr - 2 : fa.arr - 5) * nb + ((x0 * O + x1) * V + x2) * V + x3];
                }
            }
            sum += prod;
        }
        return sum;
    };
    double* C1[2] = {c1a, c1b};
    for (int s = 0; s < 2; ++s)
        for (long i = 0; i < o; ++i)
            for (long a = 0; a < v; ++a) {
                const long I = occ(s, i), A = vir(s, a);
                const long q[4] = {I, A, 0, 0};
                C1[s][i * v + a] = eval(48 + s * 4 + ((I == f.occ_act[s]) << 1) + (A == f.vir_act[s]), q);
            }
    double* C2[3] = {c2aa, c2bb, c2ab};
    for (int blk = 0; blk < 3; ++blk) {
        const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
        for (long i = 0; i < o; ++i)
            for (long j = 0; j < o; ++j)
                for (long a = 0; a < v; ++a)
                    for (long b = 0; b < v; ++b) {
                        const long I = occ(s1, i), J = occ(s2, j), A = vir(s1, a), B = vir(s2, b);
                        const bool ai = I == f.occ_act[s1], aj = J == f.occ_act[s2];
                        const bool aa = A == f.vir_act[s1], ab = B == f.vir_act[s2];
                        double cv = 0.0;
                        const bool same_spin_diag = blk != 2 && (i == j || a == b);
                        const bool a_to_b = blk == 2 && ai && aj && aa && ab;
                        if (!same_spin_diag && !a_to_b) {
                            const long q[4] = {I, J, A, B};
                            cv = eval(blk * 16 + (ai << 3) + (aj << 2) + (aa << 1) + ab, q);
                        }
                        C2[blk][((i * o + j) * v + a) * v + b] = cv;
                    }
    }
    return DCSD_OK;
}

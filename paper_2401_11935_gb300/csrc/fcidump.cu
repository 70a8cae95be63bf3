// FCIDUMP input (the integral file format the paper's calculations read,
// Section III) and its preparation for the engine: frozen-core folding, the
// Fock matrices of Phi_A, and an exact pivoted Cholesky factorisation of the
// four-index integrals, which takes the place of density fitting.  Host
// code; the factors then enter dcsd_init like DF factors.
//
// FCIDUMP (Knowles-Handy format): a namelist header "&FCI NORB=..,
// NELEC=.., MS2=.., ORBSYM=..., ISYM=.., &END" (or "/" as terminator),
// then lines "value i j k l" with 1-based orbital indices: (ij|kl) for
// i,j,k,l > 0 (chemists' notation, one representative of the eight
// permutations (ij|kl) = (ji|kl) = (ij|lk) = (kl|ij) ...), h_ij for
// k = l = 0, an orbital energy for j = k = l = 0 (ignored) and the core
// energy for i = j = k = l = 0.  Spin-restricted (ROHF, 2D-SCF) orbitals.
//
// Cholesky factorisation (Beebe and Linderberg, Int. J. Quantum Chem. 12,
// 683 (1977)): V[(pq),(rs)] = (pq|rs) is positive semidefinite; the pivoted
// Cholesky steps take the largest remaining diagonal element as pivot P,
// L_P = (V[:,P] - sum_k B_k B_k[P]) / sqrt(D[P]), D -= L_P^2, until every
// remaining diagonal element is below the threshold; then
// |(pq|rs) - sum_L B^L_pq B^L_rs| <= threshold for every element.
#include "common.h"

#include <algorithm>
#include <cctype>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

namespace {

constexpr int kMaxOrb = 160;  // dense host four-index array: 160^4 doubles = 5.2 GB

struct Header {
    int norb = -1, nelec = -1, ms2 = 0;
};

std::string upper(std::string s) {
    for (auto& ch : s) ch = (char)std::toupper((unsigned char)ch);
    return s;
}

// value of KEY=number in the header text (after the key, skipping blanks)
bool header_int(const std::string& h, const char* key, int& out) {
    const std::string k = key;
    size_t pos = 0;
    while ((pos = h.find(k, pos)) != std::string::npos) {
        // whole word: the preceding character is not a letter
        if (pos > 0 && std::isalpha((unsigned char)h[pos - 1])) {
            pos += k.size();
            continue;
        }
        size_t q = pos + k.size();
        while (q < h.size() && std::isspace((unsigned char)h[q])) ++q;
        if (q < h.size() && h[q] == '=') {
            ++q;
            while (q < h.size() && std::isspace((unsigned char)h[q])) ++q;
            char* end = nullptr;
            const long v = std::strtol(h.c_str() + q, &end, 10);
            if (end == h.c_str() + q) return false;
            out = (int)v;
            return true;
        }
        pos += k.size();
    }
    return false;
}

// Reads the header; leaves the stream at the first integral line.
bool read_header(std::ifstream& f, Header& hd, std::string& err) {
    std::string text, line;
    bool started = false;
    while (std::getline(f, line)) {
        const std::string u = upper(line);
        if (!started) {
            if (u.find("&FCI") == std::string::npos) continue;
            started = true;
        }
        text += " " + u;
        if (u.find("&END") != std::string::npos || u.find('/') != std::string::npos) break;
    }
    if (!started) {
        err = "no &FCI header";
        return false;
    }
    if (!header_int(text, "NORB", hd.norb) || !header_int(text, "NELEC", hd.nelec)) {
        err = "header lacks NORB or NELEC";
        return false;
    }
    header_int(text, "MS2", hd.ms2);
    int iuhf = 0;
    if (header_int(text, "IUHF", iuhf) && iuhf != 0) {
        err = "unrestricted (IUHF) integral files are not supported";
        return false;
    }
    return true;
}

// Fortran-style exponents (1.0D-03) are accepted
bool parse_line(std::string line, double& v, int idx[4]) {
    for (auto& ch : line)
        if (ch == 'D' || ch == 'd') ch = 'E';
    std::istringstream is(line);
    if (!(is >> v >> idx[0] >> idx[1] >> idx[2] >> idx[3])) return false;
    return true;
}

dcsd_status read_file(const char* path, Header& hd, std::vector<double>* h, std::vector<double>* eri,
                      double* ecore, std::string& err) {
    std::ifstream f(path);
    if (!f) {
        err = std::string("cannot open ") + path;
        return DCSD_ERR_INVALID_ARG;
    }
    if (!read_header(f, hd, err)) return DCSD_ERR_INVALID_ARG;
    const int n = hd.norb;
    if (n < 1 || n > kMaxOrb) {
        err = "NORB out of range (1.." + std::to_string(kMaxOrb) + ")";
        return DCSD_ERR_INVALID_ARG;
    }
    if (!h && !eri && !ecore) return DCSD_OK;
    const size_t n2 = (size_t)n * n;
    if (h) h->assign(n2, 0.0);
    if (eri) eri->assign(n2 * n2, 0.0);
    if (ecore) *ecore = 0.0;
    std::string line;
    long lineno = 0;
    while (std::getline(f, line)) {
        ++lineno;
        if (line.find_first_not_of(" \t\r") == std::string::npos) continue;
        double v;
        int q[4];
        if (!parse_line(line, v, q)) {
            err = "malformed integral line " + std::to_string(lineno) + " after the header";
            return DCSD_ERR_INVALID_ARG;
        }
        for (int k = 0; k < 4; ++k)
            if (q[k] < 0 || q[k] > n) {
                err = "orbital index out of range on integral line " + std::to_string(lineno);
                return DCSD_ERR_INVALID_ARG;
            }
        const int i = q[0] - 1, j = q[1] - 1, k = q[2] - 1, l = q[3] - 1;
        if (q[0] > 0 && q[1] > 0 && q[2] > 0 && q[3] > 0) {
            if (!eri) continue;
            const int p4[8][4] = {{i, j, k, l}, {j, i, k, l}, {i, j, l, k}, {j, i, l, k},
                                  {k, l, i, j}, {l, k, i, j}, {k, l, j, i}, {l, k, j, i}};
            for (auto& p : p4) (*eri)[((size_t)(p[0] * n + p[1]) * n + p[2]) * n + p[3]] = v;
        } else if (q[0] > 0 && q[1] > 0 && q[2] == 0 && q[3] == 0) {
            if (h) (*h)[(size_t)i * n + j] = (*h)[(size_t)j * n + i] = v;
        } else if (q[0] == 0 && q[1] == 0 && q[2] == 0 && q[3] == 0) {
            if (ecore) *ecore = v;
        }
        // orbital energies (i > 0, j = k = l = 0) are not used
    }
    return DCSD_OK;
}

// Pivoted Cholesky of V[(pq),(rs)] = eri (n^2 x n^2, row-major pairs);
// factors B[L][pq] appended to `B`.  Stops when the largest remaining
// diagonal element is <= tol or at max_rank.
void cholesky(int n, const double* eri, double tol, int max_rank, std::vector<double>& B, int& rank,
              double& max_diag_left) {
    const size_t m = (size_t)n * n;
    std::vector<double> D(m);
    for (size_t pq = 0; pq < m; ++pq) D[pq] = eri[pq * m + pq];
    B.clear();
    rank = 0;
    std::vector<double> col(m);
    while (rank < max_rank) {
        size_t P = 0;
        for (size_t pq = 1; pq < m; ++pq)
            if (D[pq] > D[P]) P = pq;
        if (!(D[P] > tol)) break;
        const double s = 1.0 / std::sqrt(D[P]);
        for (size_t rs = 0; rs < m; ++rs) {
            double x = eri[rs * m + P];
            for (int k = 0; k < rank; ++k) x -= B[(size_t)k * m + rs] * B[(size_t)k * m + P];
            col[rs] = x * s;
        }
        B.insert(B.end(), col.begin(), col.end());
        for (size_t rs = 0; rs < m; ++rs) D[rs] -= col[rs] * col[rs];
        D[P] = 0.0;
        ++rank;
    }
    max_diag_left = 0.0;
    for (size_t pq = 0; pq < m; ++pq) max_diag_left = std::max(max_diag_left, D[pq]);
}

// Everything dcsd_init needs, from an FCIDUMP file.
struct Prepared {
    dcsd_fcidump_info info{};
    std::vector<double> fa, fb, B, vvvv;  // Fock of Phi_A (alpha, beta), factors, (ac|bd) of the union virtuals
};

dcsd_status prepare(const char* path, int n_frozen, double chol_tol, bool want_vvvv, Prepared& out, std::string& err) {
    Header hd;
    std::vector<double> h, eri;
    double ecore = 0.0;
    DCSD_TRY(read_file(path, hd, &h, &eri, &ecore, err));
    const int N = hd.norb;
    if (hd.ms2 != 0 || hd.nelec < 2 || hd.nelec % 2 != 0) {
        err = "an open-shell singlet / M_s = 0 triplet needs MS2 = 0 and an even NELEC >= 2";
        return DCSD_ERR_INVALID_ARG;
    }
    const int ndocc = (hd.nelec - 2) / 2;  // doubly occupied in Phi_A, frozen ones included
    if (n_frozen < 0 || n_frozen > ndocc || ndocc + 2 >= N) {
        err = "frozen-core count or orbital counts inconsistent with NELEC/NORB (need at least one virtual)";
        return DCSD_ERR_INVALID_ARG;
    }
    if (!(chol_tol > 0.0)) {
        err = "Cholesky threshold must be positive";
        return DCSD_ERR_INVALID_ARG;
    }
    auto V4 = [&](int p, int q, int r, int s) { return eri[((size_t)(p * N + q) * N + r) * N + s]; };
    // frozen core: h'_pq = h_pq + sum_f [2 (pq|ff) - (pf|fq)],
    // E_core' = E_core + sum_f [2 h_ff] + sum_fg [2 (ff|gg) - (fg|gf)]
    const int nf = n_frozen, n = N - nf;
    double ec = ecore;
    for (int f = 0; f < nf; ++f) {
        ec += 2.0 * h[(size_t)f * N + f];
        for (int g = 0; g < nf; ++g) ec += 2.0 * V4(f, f, g, g) - V4(f, g, g, f);
    }
    std::vector<double> hp((size_t)n * n);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double x = h[(size_t)(p + nf) * N + (q + nf)];
            for (int f = 0; f < nf; ++f) x += 2.0 * V4(p + nf, q + nf, f, f) - V4(p + nf, f, f, q + nf);
            hp[(size_t)p * n + q] = x;
        }
    // correlated four-index block
    std::vector<double> e4((size_t)n * n * n * n);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q)
            for (int r = 0; r < n; ++r)
                for (int s = 0; s < n; ++s) e4[((size_t)(p * n + q) * n + r) * n + s] = V4(p + nf, q + nf, r + nf, s + nf);
    auto E4 = [&](int p, int q, int r, int s) { return e4[((size_t)(p * n + q) * n + r) * n + s]; };
    // Phi_A over the correlated orbitals: core 0..nc-1 both spins, t alpha, u beta
    const int nc = ndocc - nf, t = nc, u = nc + 1;
    std::vector<int> occ[2];
    for (int k = 0; k < nc; ++k) {
        occ[0].push_back(k);
        occ[1].push_back(k);
    }
    occ[0].push_back(t);
    occ[1].push_back(u);
    // f^sigma_pq = h'_pq + sum_{k in occ_A} [(pq|kk) - delta(sigma_k, sigma) (pk|kq)]
    out.fa.assign((size_t)n * n, 0.0);
    out.fb.assign((size_t)n * n, 0.0);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) {
            double J = 0.0, K[2] = {0.0, 0.0};
            for (int sg = 0; sg < 2; ++sg)
                for (int k : occ[sg]) {
                    J += E4(p, q, k, k);
                    K[sg] += E4(p, k, k, q);
                }
            out.fa[(size_t)p * n + q] = hp[(size_t)p * n + q] + J - K[0];
            out.fb[(size_t)p * n + q] = hp[(size_t)p * n + q] + J - K[1];
        }
    // <Phi_A|H|Phi_A> = E_core' + sum_k h'_kk + 1/2 sum_{k,l} <kl||kl>
    double eref = ec;
    for (int sg = 0; sg < 2; ++sg)
        for (int k : occ[sg]) eref += hp[(size_t)k * n + k];
    for (int s1 = 0; s1 < 2; ++s1)
        for (int k : occ[s1])
            for (int s2 = 0; s2 < 2; ++s2)
                for (int l : occ[s2]) eref += 0.5 * (E4(k, k, l, l) - (s1 == s2 ? E4(k, l, l, k) : 0.0));
    int rank = 0;
    double left = 0.0;
    cholesky(n, e4.data(), chol_tol, n * (n + 1) / 2, out.B, rank, left);
    if (rank == 0) {
        err = "the two-electron integrals are zero to the Cholesky threshold";
        return DCSD_ERR_INVALID_ARG;
    }
    // the residual matrix V - B^T B is positive semidefinite, so each of its
    // elements is bounded by the largest remaining diagonal element
    const double maxerr = left;
    if (want_vvvv) {
        // (ac|bd) over the union virtuals (t, u, external), stored [a][c][b][d]
        const int V = n - nc;
        out.vvvv.resize((size_t)V * V * V * V);
        for (int a = 0; a < V; ++a)
            for (int c = 0; c < V; ++c)
                for (int b = 0; b < V; ++b)
                    for (int d = 0; d < V; ++d)
                        out.vvvv[(((size_t)a * V + c) * V + b) * V + d] = E4(nc + a, nc + c, nc + b, nc + d);
    }
    dcsd_fcidump_info& I = out.info;
    I.norb = N;
    I.nelec = hd.nelec;
    I.ms2 = hd.ms2;
    I.n_frozen = nf;
    I.n_c = nc;
    I.n_v = n - nc - 2;
    I.naux = rank;
    I.e_core = ec;
    I.e_ref = eref;
    I.chol_max_error = maxerr;
    return DCSD_OK;
}

std::string g_fcidump_error;

}  // namespace

extern "C" dcsd_status dcsd_fcidump_header(const char* path, int* norb, int* nelec, int* ms2) {
    if (!path || !norb || !nelec || !ms2) return DCSD_ERR_INVALID_ARG;
    Header hd;
    std::string err;
    const dcsd_status st = read_file(path, hd, nullptr, nullptr, nullptr, err);
    if (st != DCSD_OK) {
        g_fcidump_error = err;
        return st;
    }
    *norb = hd.norb;
    *nelec = hd.nelec;
    *ms2 = hd.ms2;
    return DCSD_OK;
}

extern "C" dcsd_status dcsd_fcidump_read(const char* path, int norb, double* h, double* eri, double* ecore) {
    if (!path || !h || !eri || !ecore) return DCSD_ERR_INVALID_ARG;
    Header hd;
    std::vector<double> hv, ev;
    std::string err;
    const dcsd_status st = read_file(path, hd, &hv, &ev, ecore, err);
    if (st != DCSD_OK) {
        g_fcidump_error = err;
        return st;
    }
    if (hd.norb != norb) {
        g_fcidump_error = "NORB differs from the size passed";
        return DCSD_ERR_INVALID_ARG;
    }
    std::memcpy(h, hv.data(), hv.size() * sizeof(double));
    std::memcpy(eri, ev.data(), ev.size() * sizeof(double));
    return DCSD_OK;
}

extern "C" dcsd_status dcsd_cholesky_host(int n, const double* eri, double tol, int max_rank, double* B, int* rank,
                                          double* max_diag_left) {
    if (n < 1 || n > kMaxOrb || !eri || !B || !rank || !(tol > 0.0) || max_rank < 1) return DCSD_ERR_INVALID_ARG;
    std::vector<double> Bv;
    int r = 0;
    double left = 0.0;
    cholesky(n, eri, tol, max_rank, Bv, r, left);
    std::memcpy(B, Bv.data(), Bv.size() * sizeof(double));
    *rank = r;
    if (max_diag_left) *max_diag_left = left;
    return DCSD_OK;
}

extern "C" dcsd_status dcsd_fcidump_prepare(const char* path, int n_frozen, double chol_tol, dcsd_fcidump_info* info,
                                            double* fock_a, double* fock_b, double* B) {
    if (!path || !info) return DCSD_ERR_INVALID_ARG;
    Prepared p;
    std::string err;
    const dcsd_status st = prepare(path, n_frozen, chol_tol, false, p, err);
    if (st != DCSD_OK) {
        g_fcidump_error = err;
        return st;
    }
    *info = p.info;
    if (fock_a) std::memcpy(fock_a, p.fa.data(), p.fa.size() * sizeof(double));
    if (fock_b) std::memcpy(fock_b, p.fb.data(), p.fb.size() * sizeof(double));
    if (B) std::memcpy(B, p.B.data(), p.B.size() * sizeof(double));
    return DCSD_OK;
}

extern "C" const char* dcsd_fcidump_error(void) { return g_fcidump_error.c_str(); }

namespace dcsd {
dcsd_status set_vvvv(Ctx* c, const double* host_vvvv);
}

extern "C" dcsd_status dcsd_init_fcidump(dcsd_ctx** out, const char* path, int n_frozen, double chol_tol,
                                         int stored_ladder, void* stream, dcsd_fcidump_info* info) {
    if (!out || !path || (stored_ladder != 0 && stored_ladder != 1)) return DCSD_ERR_INVALID_ARG;
    *out = nullptr;
    Prepared p;
    std::string err;
    dcsd_status st = prepare(path, n_frozen, chol_tol, stored_ladder == 1, p, err);
    if (st != DCSD_OK) {
        g_fcidump_error = err;
        return st;
    }
    dcsd_dims d{p.info.n_c, p.info.n_v, p.info.naux};
    st = dcsd_init(out, &d, nullptr, p.fa.data(), p.fb.data(), p.B.data(), DCSD_MEM_HOST, stream);
    if (st != DCSD_OK) {
        g_fcidump_error = dcsd_last_error(nullptr);
        return st;
    }
    if (stored_ladder) {
        st = dcsd::set_vvvv(&(*out)->c, p.vvvv.data());
        if (st != DCSD_OK) {
            g_fcidump_error = (*out)->c.err;
            dcsd_destroy(*out);
            *out = nullptr;
            return st;
        }
    }
    if (info) *info = p.info;
    return DCSD_OK;
}

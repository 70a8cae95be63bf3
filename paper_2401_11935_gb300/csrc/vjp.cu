// Reverse mode of the FP64 residual: vector-Jacobian products
//   (R1_bar, R2_bar, dE_bar, W_bar) -> (T1_bar, T2_bar, B_bar, f_bar).
//
// The FP64 residual (residual.cu) runs once with recording switched on: every
// contraction, elementwise update, copy and custom kernel appends an entry to
// the context's tape, and each intermediate gets its own buffer from an arena
// whose twin holds its adjoint.  The reverse sweep then walks the tape
// backwards and applies each entry's adjoint:
//   C = beta C + alpha einsum(A, B):  A_bar += alpha einsum(C_bar, B),
//                                     B_bar += alpha einsum(A, C_bar),
//                                     C_bar *= beta;
//   elementwise updates, copies, zero fills and dot products likewise;
//   the T1 dressing matrices, the occupied Fock terms of the hole-hole
//   intermediate, the energy combination and the two-determinant coupling
//   terms have hand-written adjoint kernels.
// The particle-particle ladder is one tape entry: its integrals (ac|bd) are
// rebuilt chunk by chunk in the reverse sweep, never stored.  Its adjoint
// uses the symmetry (ac|bd) = (ca|db): T2_bar += ladder(R2_bar), and
// B_bar from the chunk intermediate Y[a][c][b][d] = sum_sij R2_bar[sij][ab]
// t2[sij][cd].  The integrals J = (kc|ld) and the reference exchange K built
// at initialisation are re-recorded so that their adjoints reach B_bar.
#include "common.h"

#include <algorithm>
#include <cstring>

namespace dcsd {

// ---------------------------------------------------------------------------
// recording
// ---------------------------------------------------------------------------
double* scratch(Ctx* c, double* normal, size_t elems) {
    if (!c->rec) return normal;
    const size_t need = (std::max<size_t>(elems, 1) + 31) & ~(size_t)31;  // 256-byte granules
    for (auto& b : c->arena)
        if (b.cap - b.used >= need) {
            double* p = b.fwd + b.used;
            b.used += need;
            return p;
        }
    ArenaBlock nb;
    nb.cap = std::max(need, (size_t)32 << 20);
    if (cudaMalloc((void**)&nb.fwd, nb.cap * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&nb.adj, nb.cap * sizeof(double)) != cudaSuccess ||
        cudaMemsetAsync(nb.adj, 0, nb.cap * sizeof(double), c->stream) != cudaSuccess) {
        cudaGetLastError();
        if (nb.fwd) cudaFree(nb.fwd);
        if (nb.adj) cudaFree(nb.adj);
        // keep the forward running on the shared buffer; the caller reports
        c->err = "reverse mode: arena allocation failed";
        c->rec = false;
        c->tape.clear();
        return normal;
    }
    nb.used = need;
    c->arena.push_back(nb);
    c->regions.push_back({nb.fwd, nb.cap, nb.adj});
    return nb.fwd;
}

void rec_push(Ctx* c, TapeOp&& op) { c->tape.push_back(std::move(op)); }

dcsd_status copy_dev(Ctx* c, double* dst, const double* src, size_t n) {
    if (c->rec) {
        TapeOp op;
        op.type = OP_COPY;
        op.A = view((double*)src, {(long)n});
        op.C = view(dst, {(long)n});
        rec_push(c, std::move(op));
    }
    DCSD_CUDA(c, cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return DCSD_OK;
}

dcsd_status zero_dev(Ctx* c, double* dst, size_t n) {
    if (c->rec) {
        TapeOp op;
        op.type = OP_ZERO;
        op.C = view(dst, {(long)n});
        rec_push(c, std::move(op));
    }
    DCSD_CUDA(c, cudaMemsetAsync(dst, 0, n * sizeof(double), c->stream));
    return DCSD_OK;
}

// one contraction on the engine of a precision: nsplit 0 FP64 CUDA cores,
// otherwise tensor cores with nsplit operand splits
static dcsd_status contract(Ctx* c, int nsplit, const char* spec, double alpha, const TV& A, const TV& B,
                            double beta, const TV& C) {
    if (nsplit == 0) return einsum64(c, spec, alpha, A, B, beta, C);
    return einsum_tc(c, spec, alpha, A, B, beta, C, nsplit);
}

// keeps the tensor-core packings of two operands that stay unchanged over a
// loop of contractions (t2 and B_vv in the chunked ladder and G pass)
struct PackCacheScope {
    Ctx* c;
    PackCacheScope(Ctx* c_, int nsplit, const double* s0, const double* s1) : c(nsplit > 0 ? c_ : nullptr) {
        if (c) pack_cache_set(c, s0, s1);
    }
    ~PackCacheScope() {
        if (c) pack_cache_set(c, nullptr, nullptr);
    }
};

// R2[s][ij][a][b] += sum_cd t2[s][ij][c][d] (ac|bd), (ac|bd) = sum_L B_L[a][c] B_L[b][d]
// built for chunks of `chunk` values of a in `chunkbuf` (chunk * V^3 doubles)
dcsd_status ladder64(Ctx* c, const TV& t2, const TV& Bvv, const TV& R2, double* chunkbuf, long chunk,
                     int nsplit, bool compute) {
    const long V = c->V;
    if (c->rec) {
        TapeOp op;
        op.type = OP_LADDER;
        op.A = t2;
        op.B = Bvv;
        op.C = R2;
        op.iarg[0] = (int)chunk;
        op.iarg[1] = nsplit;
        rec_push(c, std::move(op));
    }
    if (!compute) return DCSD_OK;
    const bool saved = c->rec;
    c->rec = false;
    PackCacheScope pcs(c, nsplit, t2.p, Bvv.p);
    dcsd_status st = DCSD_OK;
    for (long a0 = 0; a0 < V && st == DCSD_OK; a0 += chunk) {
        const long na = std::min(chunk, V - a0);
        TV Vc = view(chunkbuf, {na, V, V, V});  // [a][c][b][d] = (ac|bd)
        st = contract(c, nsplit, "Lac,Lbd->acbd", 1.0, sub(Bvv, 1, a0, na), Bvv, 0.0, Vc);
        if (st == DCSD_OK) st = contract(c, nsplit, "sijcd,acbd->sijab", 1.0, t2, Vc, 1.0, sub(R2, 3, a0, na));
    }
    c->rec = saved;
    return st;
}

// G[s][i][j][k][b] = sum_cd t2[s][ij][cd] (kc|bd) for s = aa, bb, ab and
// G[3][i][j][k][b] = sum_cd t2ab[ij][dc] (kc|bd), by chunks of k
dcsd_status gpass(Ctx* c, const TV& t2, const TV& Bov, const TV& Bvv, const TV& G, double* chunkbuf, long chunk,
                  int nsplit, bool compute) {
    const long O = c->O, V = c->V;
    if (c->rec) {
        TapeOp op;
        op.type = OP_GPASS;
        op.A = t2;
        op.B = Bov;
        op.X[0] = Bvv;
        op.C = G;
        op.iarg[0] = (int)chunk;
        op.iarg[1] = nsplit;
        rec_push(c, std::move(op));
    }
    if (!compute) return DCSD_OK;
    const bool saved = c->rec;
    c->rec = false;
    dcsd_status st = DCSD_OK;
    const TV t2ab = fix(t2, 0, 2);
    PackCacheScope pcs(c, nsplit, t2.p, Bvv.p);
    for (long k0 = 0; k0 < O && st == DCSD_OK; k0 += chunk) {
        const long nk = std::min(chunk, O - k0);
        TV Ic = view(chunkbuf, {nk, V, V, V});  // [k][c][b][d] = (kc|bd)
        st = contract(c, nsplit, "Lkc,Lbd->kcbd", 1.0, sub(Bov, 1, k0, nk), Bvv, 0.0, Ic);
        if (st == DCSD_OK)
            st = contract(c, nsplit, "sijcd,kcbd->sijkb", 1.0, t2, Ic, 0.0, sub(sub(G, 0, 0, 3), 3, k0, nk));
        if (st == DCSD_OK)
            st = contract(c, nsplit, "ijdc,kcbd->ijkb", 1.0, t2ab, Ic, 0.0, sub(fix(G, 0, 3), 2, k0, nk));
    }
    c->rec = saved;
    return st;
}

namespace {

// ---------------------------------------------------------------------------
// adjoint kernels
// ---------------------------------------------------------------------------
// S = 1 - tau, T = 1 + tau with tau[p][q] = t1[q][p - nc] (p virtual, q occupied)
__global__ void k_tau_adj(int n, int nc, int O, int V, const double* Sb, const double* Tb, double* t1b) {
    const long total = (long)O * V;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int q = (int)(e / V), a = (int)(e % V);
        const long pq = (long)(nc + a) * n + q;
        t1b[e] += Tb[pq] - Sb[pq];
    }
}

// Wo[k][l][i][j] -= d_ki F2[l][j] + d_lj F1[k][i]
__global__ void k_fockhh_adj(int O, const double* Wb, double* F1b, double* F2b) {
    const long total = (long)O * O;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int r = (int)(e / O), s = (int)(e % O);
        double f2 = 0.0, f1 = 0.0;
        for (int k = 0; k < O; ++k) f2 += Wb[(((long)k * O + r) * O + k) * O + s];  // F2[l=r][j=s]
        for (int l = 0; l < O; ++l) f1 += Wb[(((long)r * O + l) * O + s) * O + l];  // F1[k=r][i=s]
        if (F2b) F2b[e] -= f2;
        if (F1b) F1b[e] -= f1;
    }
}

double* adj_of(Ctx* c, const double* p) {
    for (const auto& r : c->regions)
        if (p >= r.fwd && p < r.fwd + r.len) return r.adj + (p - r.fwd);
    return nullptr;
}

bool adj_view(Ctx* c, const TV& v, TV& out) {
    double* a = adj_of(c, v.p);
    if (!a) return false;
    out = v;
    out.p = a;
    return true;
}

void split_spec(const std::string& spec, std::string& a, std::string& b, std::string& cc) {
    const size_t comma = spec.find(','), arrow = spec.find("->");
    a = spec.substr(0, comma);
    b = spec.substr(comma + 1, arrow - comma - 1);
    cc = spec.substr(arrow + 2);
}

// C_bar *= beta over a strided view
dcsd_status scale_adj(Ctx* c, const TV& Cb, double beta) {
    if (beta == 1.0) return DCSD_OK;
    return axpy_view(c, 0.0, Cb, beta, Cb);
}

dcsd_status read_scalar(Ctx* c, const double* dev, double* host) {
    DCSD_CUDA(c, cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
    return DCSD_OK;
}

dcsd_status write_scalar(Ctx* c, double* dev, double v) {
    DCSD_CUDA(c, cudaMemcpyAsync(dev, &v, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
    return DCSD_OK;
}

// Pair-row stack of a [3][O][O][V][V] array: rows 0..P-1 are the alpha-alpha
// pairs i < j (row-major), P..2P-1 the beta-beta pairs, then the O*O
// alpha-beta rows.  antisym: a pair row holds x[s][i][j] - x[s][j][i].
__device__ __forceinline__ void pair_row_index(long r, long O, long P, long& s, long& i, long& j) {
    if (r < 2 * P) {
        s = r / P;
        long p = r - s * P;
        i = 0;
        while (p >= O - 1 - i) {
            p -= O - 1 - i;
            ++i;
        }
        j = i + 1 + p;
    } else {
        s = 2;
        const long q = r - 2 * P;
        i = q / O;
        j = q - i * O;
    }
}

__global__ void k_pair_rows(long O, long VV, const double* __restrict__ x, double* __restrict__ y, int antisym) {
    const long P = O * (O - 1) / 2, R = 2 * P + O * O;
    for (long r = blockIdx.x; r < R; r += gridDim.x) {
        long s, i, j;
        pair_row_index(r, O, P, s, i, j);
        const double* a = x + ((s * O + i) * O + j) * VV;
        const double* b = x + ((s * O + j) * O + i) * VV;
        double* out = y + r * VV;
        if (antisym && s < 2)
            for (long e = threadIdx.x; e < VV; e += blockDim.x) out[e] = a[e] - b[e];
        else
            for (long e = threadIdx.x; e < VV; e += blockDim.x) out[e] = a[e];
    }
}

// x[s][i][j] += y[r] for every stacked row r
__global__ void k_pair_rows_add(long O, long VV, const double* __restrict__ y, double* __restrict__ x) {
    const long P = O * (O - 1) / 2, R = 2 * P + O * O;
    for (long r = blockIdx.x; r < R; r += gridDim.x) {
        long s, i, j;
        pair_row_index(r, O, P, s, i, j);
        double* out = x + ((s * O + i) * O + j) * VV;
        const double* in = y + r * VV;
        for (long e = threadIdx.x; e < VV; e += blockDim.x) out[e] += in[e];
    }
}

static bool is_amp_layout(const Ctx* c, const TV& v) {
    const long O = c->O, V = c->V;
    const long sz[5] = {3, O, O, V, V};
    if (v.rank != 5) return false;
    long st = 1;
    for (int k = 4; k >= 0; --k) {
        if (v.size[k] != sz[k] || v.stride[k] != st) return false;
        st *= sz[k];
    }
    return true;
}

// Reverse of the ladder on the tensor cores.  The recorded forward (the fused
// tensor-core ladder) reads the same-spin amplitudes only at i < j and writes
// R2[ij] and R2[ji] = -R2[ij] from them, so its adjoint contracts pair rows:
// t2_bar[ij] += L^T (R2_bar[ij] - R2_bar[ji]) for i < j (nothing for i > j),
// and Y = sum_ij t2[ij] R2_bar[ij] = sum_{i<j} t2[ij] (R2_bar[ij] - R2_bar[ji]).
// Returns false (nothing done) when the pair-row buffers cannot be had.
static bool ladder_reverse_pairs(Ctx* c, const TapeOp& op, const TV& R2b, bool want_t, const TV& t2b, bool want_B,
                                 const TV& Bvvb, dcsd_status& st) {
    const long O = c->O, V = c->V, VV = V * V, chunk = op.iarg[0];
    const int ns = op.iarg[1];
    if (!is_amp_layout(c, op.A) || !is_amp_layout(c, R2b) || (want_t && !is_amp_layout(c, t2b))) return false;
    const long Rr = O * (O - 1) + O * O;
    const size_t need = (size_t)3 * Rr * VV;
    if (c->pairbuf_elems < need) {
        if (c->pairbuf) cudaFree(c->pairbuf);
        c->pairbuf = nullptr;
        c->pairbuf_elems = 0;
        if (cudaMalloc((void**)&c->pairbuf, need * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        c->pairbuf_elems = need;
    }
    double* Tt = c->pairbuf;            // pair rows of t2
    double* Rt = Tt + (size_t)Rr * VV;  // antisymmetrised pair rows of R2_bar
    double* Tb = Rt + (size_t)Rr * VV;  // adjoint of the pair rows of t2
    const unsigned g = (unsigned)std::max<long>(1, std::min<long>(Rr, (long)c->num_sms * 4));
    st = DCSD_OK;
    k_pair_rows<<<g, 256, 0, c->stream>>>(O, VV, R2b.p, Rt, 1);
    if ((st = launch_check(c, "pair_rows")) != DCSD_OK) return true;
    if (want_B) {
        k_pair_rows<<<g, 256, 0, c->stream>>>(O, VV, op.A.p, Tt, 0);
        if ((st = launch_check(c, "pair_rows")) != DCSD_OK) return true;
    }
    if (want_t && cudaMemsetAsync(Tb, 0, (size_t)Rr * VV * sizeof(double), c->stream) != cudaSuccess) {
        cudaGetLastError();
        c->err = "reverse mode: cudaMemsetAsync of the pair-row adjoint failed";
        st = DCSD_ERR_CUDA;
        return true;
    }
    const TV Ttv = view(Tt, {Rr, V, V}), Rtv = view(Rt, {Rr, V, V}), Tbv = view(Tb, {Rr, V, V});
    PackCacheScope pcs(c, ns, Tt, op.B.p);
    for (long a0 = 0; a0 < V && st == DCSD_OK; a0 += chunk) {
        const long na = std::min(chunk, V - a0);
        if (want_t) {
            TV Vc = view(c->big0, {na, V, V, V});
            if ((st = contract(c, ns, "Lac,Lbd->acbd", 1.0, sub(op.B, 1, a0, na), op.B, 0.0, Vc)) != DCSD_OK) break;
            if ((st = contract(c, ns, "rab,acbd->rcd", 1.0, sub(Rtv, 1, a0, na), Vc, 1.0, Tbv)) != DCSD_OK) break;
        }
        if (want_B) {
            // rows of S = Y + Y^T (see the all-rows form in reverse_op), then B_bar += B S
            TV Yc = view(c->big1, {na, V, V, V});
            if ((st = contract(c, ns, "rcd,rab->acbd", 1.0, Ttv, sub(Rtv, 1, a0, na), 0.0, Yc)) != DCSD_OK) break;
            if ((st = contract(c, ns, "rdc,rba->acbd", 1.0, Ttv, sub(Rtv, 2, a0, na), 1.0, Yc)) != DCSD_OK) break;
            if ((st = contract(c, ns, "Lac,acbd->Lbd", 1.0, sub(op.B, 1, a0, na), Yc, 1.0, Bvvb)) != DCSD_OK) break;
        }
    }
    if (st == DCSD_OK && want_t) {
        k_pair_rows_add<<<g, 256, 0, c->stream>>>(O, VV, Tb, t2b.p);
        st = launch_check(c, "pair_rows_add");
    }
    return true;
}

__global__ void k_ccond_adj(const double* t1, double* t1b, double* t2be, long p, long q) {
    const double g = *t2be;
    t1b[p] -= t1[q] * g;
    t1b[q] -= t1[p] * g;
    *t2be = 0.0;
}

__global__ void k_wfull_adj(const double* scal, double* sb, const double* t1, double* t1b, double* R1b, double* R2be,
                            long p, long q) {
    const double g = sb[0];
    const double r1p = scal[50], r1q = scal[51];
    if (R2be) *R2be += g;
    if (t1b) {
        t1b[p] += g * r1q;
        t1b[q] += g * r1p;
    }
    if (R1b) {
        R1b[q] += g * t1[p];
        R1b[p] += g * t1[q];
    }
    sb[0] = 0.0;
}

dcsd_status reverse_op(Ctx* c, const TapeOp& op) {
    TV Ab, Bb, Cb;
    switch (op.type) {
        case OP_EINSUM: {
            if (!adj_view(c, op.C, Cb)) return DCSD_OK;
            std::string sa, sb, sc;
            split_spec(op.spec, sa, sb, sc);
            auto run = [&](const std::string& sp, const TV& x, const TV& y, const TV& z) -> dcsd_status {
                if (op.iarg[1] == 1) return einsum32(c, sp.c_str(), op.alpha, x, y, 1.0, z);
                if (op.iarg[1] == 2) return einsum_tc(c, sp.c_str(), op.alpha, x, y, 1.0, z, op.iarg[2]);
                return einsum64(c, sp.c_str(), op.alpha, x, y, 1.0, z);
            };
            if (adj_view(c, op.A, Ab)) DCSD_TRY(run(sc + "," + sb + "->" + sa, Cb, op.B, Ab));
            if (adj_view(c, op.B, Bb)) DCSD_TRY(run(sa + "," + sc + "->" + sb, op.A, Cb, Bb));
            return scale_adj(c, Cb, op.beta);
        }
        case OP_AXPY: {
            if (!adj_view(c, op.C, Cb)) return DCSD_OK;
            if (adj_view(c, op.A, Ab)) DCSD_TRY(axpy_view(c, op.alpha, Cb, 1.0, Ab));
            return scale_adj(c, Cb, op.beta);
        }
        case OP_AXPY4: {
            if (!adj_view(c, op.C, Cb)) return DCSD_OK;
            for (int k = 0; k < op.nv; ++k) {
                TV Xb;
                if (adj_view(c, op.X[k], Xb)) DCSD_TRY(axpy_view(c, op.al[k], Cb, 1.0, Xb));
            }
            return DCSD_OK;
        }
        case OP_COPY: {
            if (!adj_view(c, op.C, Cb)) return DCSD_OK;
            if (adj_view(c, op.A, Ab)) DCSD_TRY(axpy_view(c, 1.0, Cb, 1.0, Ab));
            return scale_adj(c, Cb, 0.0);
        }
        case OP_ZERO: {
            if (!adj_view(c, op.C, Cb)) return DCSD_OK;
            return scale_adj(c, Cb, 0.0);
        }
        case OP_DOT: {
            double* ob = adj_of(c, op.p[0]);
            if (!ob) return DCSD_OK;
            double g = 0.0;
            DCSD_TRY(read_scalar(c, ob, &g));
            if (g != 0.0) {
                if (adj_view(c, op.A, Ab)) DCSD_TRY(axpy_view(c, g, op.B, 1.0, Ab));
                if (adj_view(c, op.B, Bb)) DCSD_TRY(axpy_view(c, g, op.A, 1.0, Bb));
            }
            return write_scalar(c, ob, op.beta * g);
        }
        case OP_TAU: {
            double* Sb = adj_of(c, op.A.p);
            double* Tb = adj_of(c, op.B.p);
            double* t1b = adj_of(c, c->t1 + (long)op.iarg[0] * c->O * c->V);
            if (!Sb || !Tb || !t1b) return DCSD_OK;
            k_tau_adj<<<(unsigned)std::max(1, c->num_sms * 4), 256, 0, c->stream>>>(c->n, c->nc, c->O, c->V, Sb,
                                                                                    Tb, t1b);
            return launch_check(c, "tau_adj");
        }
        case OP_FOCKHH: {
            double* Wb = adj_of(c, op.C.p);
            if (!Wb) return DCSD_OK;
            k_fockhh_adj<<<(unsigned)std::max(1, c->num_sms * 4), 256, 0, c->stream>>>(
                c->O, Wb, adj_of(c, op.A.p), adj_of(c, op.B.p));
            return launch_check(c, "fockhh_adj");
        }
        case OP_ECOMB: {
            // s1' = s1 + (s2 + s5 - s6 + s3 + s7 - s8) / 2 + s4 + s9
            double* sb = adj_of(c, c->scal);
            double h[10];
            DCSD_CUDA(c, cudaMemcpyAsync(h, sb, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
            DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
            const double g = h[1];
            h[2] += 0.5 * g; h[3] += 0.5 * g; h[5] += 0.5 * g; h[6] -= 0.5 * g;
            h[7] += 0.5 * g; h[8] -= 0.5 * g; h[4] += g; h[9] += g;
            DCSD_CUDA(c, cudaMemcpyAsync(sb, h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
            DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
            return DCSD_OK;
        }
        case OP_CCOND: {
            // t2[e] = -t1[p] t1[q]: t1b[p] -= t1[q] t2b[e], t1b[q] -= t1[p] t2b[e], t2b[e] = 0
            double* t1b = adj_of(c, c->t1);
            double* t2b = adj_of(c, c->t2);
            if (!t1b || !t2b) return DCSD_OK;
            k_ccond_adj<<<1, 1, 0, c->stream>>>(c->t1, t1b, t2b + op.pos[0], op.pos[1], op.pos[2]);
            return launch_check(c, "ccond_adj");
        }
        case OP_WFULL: {
            // W = R2[e] + t1[p] R1[q] + t1[q] R1[p] with R1[p], R1[q] saved in scal[50..51]
            double* sb = adj_of(c, c->scal);
            double* t1b = adj_of(c, c->t1);
            double* R1b = adj_of(c, c->R1);
            double* R2b = adj_of(c, c->R2);
            if (!sb) return DCSD_OK;
            k_wfull_adj<<<1, 1, 0, c->stream>>>(c->scal, sb, c->t1, t1b, R1b, R2b ? R2b + op.pos[0] : nullptr,
                                                 op.pos[1], op.pos[2]);
            return launch_check(c, "wfull_adj");
        }
        case OP_SWAPVIR:
            return swap_vir_adjoint(c, adj_of(c, c->t2s), adj_of(c, c->t2));
        case OP_MTERMS:
            return mterms_adjoint(c, op.iarg[0], adj_of(c, c->t1), adj_of(c, c->t2), adj_of(c, c->t2s),
                                  adj_of(c, c->c1), adj_of(c, c->R1), adj_of(c, c->R2), adj_of(c, c->scal));
        case OP_LADDER: {
            const long V = c->V, chunk = op.iarg[0];
            TV t2b, Bvvb, R2b;
            if (!adj_view(c, op.C, R2b)) return DCSD_OK;
            const bool want_t = adj_view(c, op.A, t2b), want_B = adj_view(c, op.B, Bvvb);
            if (op.iarg[1] > 0) {
                dcsd_status st = DCSD_OK;
                if (ladder_reverse_pairs(c, op, R2b, want_t, t2b, want_B, Bvvb, st)) return st;
            }
            PackCacheScope pcs(c, op.iarg[1], op.A.p, op.B.p);
            for (long a0 = 0; a0 < V; a0 += chunk) {
                const long na = std::min(chunk, V - a0);
                TV Vc = view(c->big0, {na, V, V, V});
                TV R2c = sub(R2b, 3, a0, na);
                const int ns = op.iarg[1];
                if (want_t) {
                    DCSD_TRY(contract(c, ns, "Lac,Lbd->acbd", 1.0, sub(op.B, 1, a0, na), op.B, 0.0, Vc));
                    DCSD_TRY(contract(c, ns, "sijab,acbd->sijcd", 1.0, R2c, Vc, 1.0, t2b));
                }
                if (want_B) {
                    // Y[a][c][b][d] = sum_sij t2[sij][cd] R2_bar[sij][ab] as a matrix over the
                    // pairs (ac), (bd); B_bar_L = B_L (Y + Y^T).  FP64 takes the two products
                    // B_L Y and B_L Y^T from the chunk rows of Y (fewer operations); the
                    // tensor cores form the rows of S = Y + Y^T instead (one long-K product
                    // less, and every product keeps a large output)
                    TV Yc = view(c->big1, {na, V, V, V});  // [a][c][b][d]
                    DCSD_TRY(contract(c, ns, "sijcd,sijab->acbd", 1.0, op.A, R2c, 0.0, Yc));
                    if (ns == 0) {
                        DCSD_TRY(contract(c, ns, "acbd,Lbd->Lac", 1.0, Yc, op.B, 1.0, sub(Bvvb, 1, a0, na)));
                    } else {
                        // Y^T rows: Y[b][d][a][c] = sum_sij t2[sij][dc] R2_bar[sij][ba]
                        DCSD_TRY(contract(c, ns, "sijdc,sijba->acbd", 1.0, op.A, sub(R2b, 4, a0, na), 1.0, Yc));
                    }
                    DCSD_TRY(contract(c, ns, "Lac,acbd->Lbd", 1.0, sub(op.B, 1, a0, na), Yc, 1.0, Bvvb));
                }
            }
            return DCSD_OK;
        }
        case OP_GPASS: {
            // G = t2 . Ic with Ic[k][c][b][d] = (kc|bd) = sum_L Bov_L[k][c] Bvv_L[b][d]
            const long O = c->O, V = c->V, chunk = op.iarg[0];
            const int ns = op.iarg[1];
            TV Gb, t2b, Bovb, Bvvb;
            if (!adj_view(c, op.C, Gb)) return DCSD_OK;
            const bool want_t = adj_view(c, op.A, t2b);
            const bool want_ov = adj_view(c, op.B, Bovb), want_vv = adj_view(c, op.X[0], Bvvb);
            const TV t2ab = fix(op.A, 0, 2);
            PackCacheScope pcs(c, ns, op.A.p, op.X[0].p);
            for (long k0 = 0; k0 < O; k0 += chunk) {
                const long nk = std::min(chunk, O - k0);
                TV Ic = view(c->big0, {nk, V, V, V});
                TV G3 = sub(sub(Gb, 0, 0, 3), 3, k0, nk), G1 = sub(fix(Gb, 0, 3), 2, k0, nk);
                DCSD_TRY(contract(c, ns, "Lkc,Lbd->kcbd", 1.0, sub(op.B, 1, k0, nk), op.X[0], 0.0, Ic));
                if (want_t) {
                    DCSD_TRY(contract(c, ns, "sijkb,kcbd->sijcd", 1.0, G3, Ic, 1.0, t2b));
                    DCSD_TRY(contract(c, ns, "ijkb,kcbd->ijdc", 1.0, G1, Ic, 1.0, fix(t2b, 0, 2)));
                }
                if (want_ov || want_vv) {
                    TV Ib = view(c->big1, {nk, V, V, V});
                    DCSD_TRY(contract(c, ns, "sijcd,sijkb->kcbd", 1.0, op.A, G3, 0.0, Ib));
                    DCSD_TRY(contract(c, ns, "ijdc,ijkb->kcbd", 1.0, t2ab, G1, 1.0, Ib));
                    if (want_ov)
                        DCSD_TRY(contract(c, ns, "kcbd,Lbd->Lkc", 1.0, Ib, op.X[0], 1.0, sub(Bovb, 1, k0, nk)));
                    if (want_vv)
                        DCSD_TRY(contract(c, ns, "Lkc,kcbd->Lbd", 1.0, sub(op.B, 1, k0, nk), Ib, 1.0, Bvvb));
                }
            }
            // the forward wrote G with beta 0
            return scale_adj(c, Gb, 0.0);
        }
        default:
            c->err = "reverse mode: unknown tape entry";
            return DCSD_ERR_INVALID_ARG;
    }
}

}  // namespace

void vjp_free(Ctx* c) {
    for (auto& b : c->arena) {
        if (b.fwd) cudaFree(b.fwd);
        if (b.adj) cudaFree(b.adj);
    }
    c->arena.clear();
    c->regions.clear();
    c->tape.clear();
    if (c->vbuf) cudaFree(c->vbuf);
    c->vbuf = nullptr;
    c->vbuf_elems = 0;
    if (c->pairbuf) cudaFree(c->pairbuf);
    c->pairbuf = nullptr;
    c->pairbuf_elems = 0;
}

// Adjoint buffers of the inputs and outputs, in the context's vbuf
struct VjpBufs {
    double *u1, *u2;  // union-layout seeds (not cleared by a sweep)
    double *t1b, *t2b, *t2sb, *c1b, *R1b, *R2b, *Bbar, *F0b, *F1b, *Jb, *Kb[4], *sb;
    size_t total, adj_elems;  // all; the adjoint part from t1b on
};

static VjpBufs vjp_layout(Ctx* c, double* base) {
    const long n = c->n, O = c->O, V = c->V, X = c->X;
    const size_t n1 = 2ul * O * V, n2 = 3ul * O * O * V * V, nn = (size_t)n * n;
    VjpBufs v;
    double* q = base;
    auto take = [&](size_t k) { double* p = q; q += k; return p; };
    v.u1 = take(n1); v.u2 = take(n2);
    v.t1b = take(n1); v.t2b = take(n2); v.t2sb = take(n2); v.c1b = take(n1); v.R1b = take(n1);
    v.R2b = take(n2); v.Bbar = take((size_t)X * nn); v.F0b = take(nn); v.F1b = take(nn);
    v.Jb = take((size_t)O * O * V * V);
    for (int k = 0; k < 4; ++k) v.Kb[k] = take(nn);
    v.sb = take(64);
    v.total = (size_t)(q - base);
    v.adj_elems = (size_t)(q - v.t1b);
    return v;
}

// Record the FP64 residual at the amplitudes already in c->t1/c->t2 and set
// up the adjoint regions.  On return the tape holds the forward.
dcsd_status vjp_record(Ctx* c, int ref, int method, int prec) {
    const long n = c->n, O = c->O, V = c->V, X = c->X;
    const size_t n1 = 2ul * O * V, n2 = 3ul * O * O * V * V, nn = (size_t)n * n;
    const size_t need = vjp_layout(c, nullptr).total;
    if (c->vbuf_elems < need) {
        if (c->vbuf) cudaFree(c->vbuf);
        c->vbuf = nullptr;
        c->vbuf_elems = 0;
        if (cudaMalloc((void**)&c->vbuf, need * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            c->err = "reverse mode: cudaMalloc of the adjoint buffers failed";
            return DCSD_ERR_OOM;
        }
        c->vbuf_elems = need;
    }
    const VjpBufs v = vjp_layout(c, c->vbuf);
    c->regions.clear();
    c->regions.push_back({c->t1, n1, v.t1b});
    c->regions.push_back({c->t2, n2, v.t2b});
    c->regions.push_back({c->t2s, n2, v.t2sb});
    c->regions.push_back({c->c1, n1, v.c1b});
    c->regions.push_back({c->R1, n1, v.R1b});
    c->regions.push_back({c->R2, n2, v.R2b});
    c->regions.push_back({c->B, (size_t)X * nn, v.Bbar});
    c->regions.push_back({c->fock[0], nn, v.F0b});
    c->regions.push_back({c->fock[1], nn, v.F1b});
    c->regions.push_back({c->J, (size_t)O * O * V * V, v.Jb});
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) c->regions.push_back({c->Kref[r][s], nn, v.Kb[2 * r + s]});
    c->regions.push_back({c->scal, 64, v.sb});
    for (auto& b : c->arena) {
        b.used = 0;
        c->regions.push_back({b.fwd, b.cap, b.adj});
    }
    c->tape.clear();
    c->rec = true;
    c->err.clear();
    struct RecGuard {
        Ctx* c;
        ~RecGuard() { c->rec = false; }
    } guard{c};
    dcsd_status st = init_constants(c, prec);
    if (st == DCSD_OK) st = residual_union(c, ref, method, prec);
    const bool lost = !c->rec;  // an arena allocation failed
    c->rec = false;
    if (st != DCSD_OK) return st;
    if (lost) return DCSD_ERR_OOM;
    return DCSD_OK;
}

// One reverse sweep over the recorded tape with seeds R_bar (union layout,
// NULL = zero), dEA_bar and W_bar; the adjoints are left in vbuf.
dcsd_status vjp_sweep(Ctx* c, const double* R1bar_u, const double* R2bar_u, double Ebar, double Wbar) {
    const size_t n1 = 2ul * c->O * c->V, n2 = 3ul * c->O * c->O * c->V * c->V;
    const VjpBufs v = vjp_layout(c, c->vbuf);
    DCSD_CUDA(c, cudaMemsetAsync(v.t1b, 0, v.adj_elems * sizeof(double), c->stream));
    for (auto& b : c->arena)
        if (b.used) DCSD_CUDA(c, cudaMemsetAsync(b.adj, 0, b.used * sizeof(double), c->stream));
    if (R1bar_u) DCSD_CUDA(c, cudaMemcpyAsync(v.R1b, R1bar_u, n1 * sizeof(double), cudaMemcpyDeviceToDevice,
                                              c->stream));
    if (R2bar_u) DCSD_CUDA(c, cudaMemcpyAsync(v.R2b, R2bar_u, n2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                              c->stream));
    {
        double* h = c->hostbuf + 40;  // pinned staging
        h[0] = Wbar;
        h[1] = Ebar;
        DCSD_CUDA(c, cudaMemcpyAsync(v.sb, h, 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    static const char* const kRevLabel[] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, "rev tau",
                                            "rev fockhh", "rev ecomb", "rev swap_vir", "rev mterms"};
    for (size_t k = c->tape.size(); k-- > 0;) {
        const TapeOp& op = c->tape[k];
        // adjoint kernels outside the traced primitives (einsum, axpy, dot)
        const char* label = (size_t)op.type < sizeof(kRevLabel) / sizeof(kRevLabel[0]) ? kRevLabel[op.type]
                                                                                       : nullptr;
        if (c->trace && label) trace_begin(c, label);
        const dcsd_status st = reverse_op(c, op);
        if (c->trace && label) trace_end(c);
        DCSD_TRY(st);
    }
    return DCSD_OK;
}

double* vjp_t1bar(Ctx* c) { return vjp_layout(c, c->vbuf).t1b; }
double* vjp_t2bar(Ctx* c) { return vjp_layout(c, c->vbuf).t2b; }
double* vjp_fbar(Ctx* c, int spin) { return spin == 0 ? vjp_layout(c, c->vbuf).F0b : vjp_layout(c, c->vbuf).F1b; }

// One VJP.  Td: device ABI amplitudes; Rb: device ABI residual cotangents
// (NULL = zero); Tb: device ABI outputs; Bb, Fab, Fbb: device outputs or NULL.
dcsd_status vjp_run(Ctx* c, int ref, int method, int prec, const double* const* Td, const double* const* Rb,
                    double Ebar, double Wbar, double* const* Tb, double* Bb, double* Fab, double* Fbb) {
    const long n = c->n, X = c->X;
    const size_t nn = (size_t)n * n;
    DCSD_TRY(unpack_T(c, ref, Td[0], Td[1], Td[2], Td[3], Td[4]));
    DCSD_TRY(vjp_record(c, ref, method, prec));
    const VjpBufs v = vjp_layout(c, c->vbuf);
    // the residual seeds in the union layout
    const double* s1 = nullptr;
    const double* s2 = nullptr;
    if (Rb) {
        double* u1 = v.u1;
        double* u2 = v.u2;
        DCSD_CUDA(c, cudaMemsetAsync(u1, 0, 2ul * c->O * c->V * sizeof(double), c->stream));
        DCSD_CUDA(c, cudaMemsetAsync(u2, 0, 3ul * c->O * c->O * c->V * c->V * sizeof(double), c->stream));
        double* Rbu[5];
        for (int k = 0; k < 5; ++k) Rbu[k] = (double*)Rb[k];
        DCSD_TRY(layout_union(c, ref, 0, u1, u2, Rbu));
        s1 = u1;
        s2 = u2;
    }
    DCSD_TRY(vjp_sweep(c, s1, s2, Ebar, Wbar));
    c->tape.clear();
    DCSD_TRY(layout_union(c, ref, 1, v.t1b, v.t2b, Tb));
    if (Bb) DCSD_CUDA(c, cudaMemcpyAsync(Bb, v.Bbar, (size_t)X * nn * sizeof(double), cudaMemcpyDeviceToDevice,
                                         c->stream));
    if (Fab) DCSD_CUDA(c, cudaMemcpyAsync(Fab, v.F0b, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    if (Fbb) DCSD_CUDA(c, cudaMemcpyAsync(Fbb, v.F1b, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
    return DCSD_OK;
}

}  // namespace dcsd

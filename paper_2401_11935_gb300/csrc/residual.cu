// One evaluation of the 2D-CCSD / 2D-DCSD residual on the GPU.
//
// Paper: arXiv 2401.11935, Section II, Eqs. 2-4.  The single-reference part
// R^X (CCSD or DCSD) is evaluated in the T1-similarity-transformed
// ("dressed") Hamiltonian, where the CCSD doubles take the form of the CCD
// doubles with dressed integrals and the singles need only T2 and dressed
// quantities:
//   Bd^s = (1 - tau^s) B (1 + tau^s)          tau^s[vir a][occ k] = t1^s[k][a]
//   fd^s = (1 - tau^s)(f^s + K^s + J(t1))(1 + tau^s) - Kd^s
// Layout: every amplitude/residual block lives on the spin-free "union"
// index spaces occ' = (core, t, u), vir' = (t, u, V), zero-padded where an
// orbital does not belong to the spin's space.  All integrals are then
// spin-free spatial quantities and the three doubles blocks (aa, bb, ab) are
// stacked rows of one matrix -- the particle-particle ladder uses one
// undressed (ac|bd) for all three blocks, plus explicit T1 corrections.
//
// DC (Section II: DC applied to the doubles as in single-reference DCSD): the
// exchange part of the quadratic ring is dropped (x = 0) and the two
// Fock-like quadratic terms are halved (y = 1/2); CCSD has x = y = 1.
//
// Fixed-reference (FR) methods (the approach of the paper's introduction):
// the A->B doubles amplitude is held at +1 (singlet) or -1 (M_s = 0
// triplet), the other amplitudes obey the single-reference equations, and
// the M W coupling terms are absent.
#include "common.h"

namespace dcsd {

namespace {

struct Views {
    long n, nc, O, V, X;
    TV B, Bov, Bvv, t1, t2, R1, R2, Bd, Z, J;
};

TV blk(const TV& v, int b) { return fix(v, 0, b); }

}  // namespace

dcsd_status init_constants(Ctx* c, int prec) {
    const long n = c->n, nc = c->nc, O = c->O, V = c->V, X = c->X;
    TV B = view(c->B, {X, n, n});
    TV Bov = sub(sub(B, 1, 0, O), 2, nc, V);
    // while recording, J and K_ref already hold these products of the same B
    // (the tensor-core precisions take the adjoints of the two large products,
    // J and the core part of K_ref, on the tensor cores)
    const bool rec = c->rec;
    const int nsplit = prec == DCSD_PREC_BF16X6 ? 3 : prec == DCSD_PREC_BF16X3 ? 2 : 1;
    auto ein = [&](const char* spec, const TV& A, const TV& Bm, double beta, const TV& C, bool tc) -> dcsd_status {
        if (!rec) return einsum64(c, spec, 1.0, A, Bm, beta, C);
        record_einsum(c, spec, 1.0, A, Bm, beta, C, tc ? 2 : 0, tc ? nsplit : 0);
        return DCSD_OK;
    };
    DCSD_TRY(ein("Lkc,Lld->klcd", Bov, Bov, 0.0, view(c->J, {O, O, V, V}), prec != DCSD_PREC_FP64));
    for (int ref = 0; ref < 2; ++ref) {
        Frame f = frame_of(c, ref);
        for (int s = 0; s < 2; ++s) {
            TV K = view(c->Kref[ref][s], {n, n});
            double beta = 0.0;
            if (nc > 0) {
                DCSD_TRY(ein("Lpk,Lkq->pq", sub(B, 2, 0, nc), sub(B, 1, 0, nc), 0.0, K, prec != DCSD_PREC_FP64));
                beta = 1.0;
            }
            DCSD_TRY(ein("Lp,Lq->pq", fix(B, 2, f.occ_act[s]), fix(B, 1, f.occ_act[s]), beta, K, false));
        }
    }
    return DCSD_OK;
}

__global__ void k_add_fock_hh(int O, double* Wo, const double* F1, const double* F2) {
    const long total = (long)O * O * O * O;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
         e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e % O), i = (int)((e / O) % O), l = (int)((e / O / O) % O),
                  k = (int)(e / O / O / O);
        double d = 0.0;
        if (k == i) d += F2[l * O + j];
        if (l == j) d += F1[k * O + i];
        Wo[e] -= d;
    }
}

dcsd_status add_fock_hh(Ctx* c, double* Wo, const double* F1, const double* F2) {
    if (c->rec) {
        TapeOp op;
        op.type = OP_FOCKHH;
        const long O = c->O;
        op.C = view(Wo, {O, O, O, O});
        op.A = view((double*)F1, {O, O});
        op.B = view((double*)F2, {O, O});
        rec_push(c, std::move(op));
    }
    const long total = (long)c->O * c->O * c->O * c->O;
    k_add_fock_hh<<<(unsigned)std::max<long>(1, std::min<long>((total + 255) / 256, 4096)), 256, 0,
                    c->stream>>>(c->O, Wo, F1, F2);
    return launch_check(c, "add_fock_hh");
}

__global__ void k_energy_combine(double* s) {
    // s[1] = f.t1 ; s[2..4] = J.t2 (aa, bb, ab); s[5..6] direct/exchange t1 t1 (aa);
    // s[7..8] (bb); s[9] ab direct
    s[1] = s[1] + 0.5 * (s[2] + s[5] - s[6] + s[3] + s[7] - s[8]) + s[4] + s[9];
}

__global__ void __launch_bounds__(256) k_merge_r2f(long n, const float* __restrict__ f, double* __restrict__ R) {
    const long stride = (long)gridDim.x * blockDim.x;
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    for (; e + stride < n; e += 2 * stride) {
        const float f0 = f[e], f1 = f[e + stride];
        const double r0 = R[e], r1 = R[e + stride];
        R[e] = r0 + f32_to_f64(f0);
        R[e + stride] = r1 + f32_to_f64(f1);
    }
    if (e < n) R[e] += f32_to_f64(f[e]);
}

dcsd_status merge_r2f(Ctx* c) {
    const long n = 3l * c->O * c->O * c->V * c->V;
    trace_begin(c, "merge_r2f");
    k_merge_r2f<<<(unsigned)std::max(1, c->num_sms * 8), 256, 0, c->stream>>>(n, c->r2f, c->R2);
    trace_end(c);
    return launch_check(c, "merge_r2f");
}

__global__ void k_c_condition(double* t2e, const double* t1s1, const double* t1s2) { *t2e = -(*t1s1) * (*t1s2); }

dcsd_status apply_c_condition(Ctx* c, int ref) {
    const InternalPos p = internal_pos(c, ref);
    if (c->rec) {
        TapeOp op;
        op.type = OP_CCOND;
        op.pos[0] = p.e;
        op.pos[1] = p.s1;
        op.pos[2] = p.s2;
        rec_push(c, std::move(op));
    }
    k_c_condition<<<1, 1, 0, c->stream>>>(c->t2 + p.e, c->t1 + p.s1, c->t1 + p.s2);
    return launch_check(c, "c_condition");
}

// W and the two singles residuals it used (kept for the reverse mode)
__global__ void k_coupling_w(double* scal, const double* R2e, const double* t1, const double* R1, long s1, long s2) {
    const double r1 = R1[s1], r2 = R1[s2];
    scal[0] = *R2e + t1[s1] * r2 + t1[s2] * r1;
    scal[50] = r1;
    scal[51] = r2;
}

dcsd_status coupling_w(Ctx* c, int ref) {
    const InternalPos p = internal_pos(c, ref);
    if (c->rec) {
        TapeOp op;
        op.type = OP_WFULL;
        op.pos[0] = p.e;
        op.pos[1] = p.s1;
        op.pos[2] = p.s2;
        rec_push(c, std::move(op));
    }
    k_coupling_w<<<1, 1, 0, c->stream>>>(c->scal, c->R2 + p.e, c->t1, c->R1, p.s1, p.s2);
    return launch_check(c, "coupling_w");
}

dcsd_status set_vvvv(Ctx* c, const double* host_vvvv) {
    const size_t V = c->V, nv4 = V * V * V * V;
    if (!c->vvvv && cudaMalloc((void**)&c->vvvv, nv4 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->vvvv = nullptr;
        c->err = "cudaMalloc of the stored (ac|bd) integrals failed";
        return DCSD_ERR_OOM;
    }
    DCSD_CUDA(c, cudaMemcpy(c->vvvv, host_vvvv, nv4 * sizeof(double), cudaMemcpyHostToDevice));
    return DCSD_OK;
}

dcsd_status residual_union(Ctx* c, int ref, int method, int prec) {
    const long n = c->n, nc = c->nc, O = c->O, V = c->V, X = c->X;
    const double x = method_dc(method) ? 0.0 : 1.0;
    const double y = method_dc(method) ? 0.5 : 1.0;
    const Frame fr = frame_of(c, ref);
    const int nsplit = prec == DCSD_PREC_BF16X6 ? 3 : prec == DCSD_PREC_BF16X3 ? 2 : 1;
    auto big = [&](const char* spec, double alpha, const TV& A, const TV& Bm, double beta,
                   const TV& C) -> dcsd_status {
        if (prec == DCSD_PREC_FP64) return einsum64(c, spec, alpha, A, Bm, beta, C);
        return einsum_tc(c, spec, alpha, A, Bm, beta, C, nsplit);
    };
    // BF16 and BF16X3 take FP32 shortcuts around the tensor cores (FP32 shadow
    // accumulation of R2, FP32 small contractions, coupling terms and Jacobi
    // step); BF16X6, the refinement precision, keeps those FP64
    const bool fast = prec == DCSD_PREC_BF16 || prec == DCSD_PREC_BF16X3;
    // small contractions: FP64 in the FP64 mode; in the fast tensor-core modes
    // the contraction engine picks the tensor cores (split-K when the output
    // is small) or, for tiny or batched shapes, FP32 products on the CUDA
    // cores (the FP64 units of this GPU run at a small fraction of its FP32
    // rate); in BF16X6 large unbatched ones (>= 4 GFLOP) go to the tensor
    // cores and the rest stay FP64
    auto sml = [&](const char* spec, double alpha, const TV& A, const TV& Bm, double beta,
                   const TV& C) -> dcsd_status {
        if (prec != DCSD_PREC_FP64 && !fast) {
            GemmPlan p;
            std::string e;
            if (plan_einsum(spec, A, Bm, C, p, e) && p.NB == 1 && p.K >= 16 &&
                2.0 * (double)p.M * (double)p.N * (double)p.K >= 4e9)
                return einsum_tc(c, spec, alpha, A, Bm, beta, C, nsplit);
            return einsum64(c, spec, alpha, A, Bm, beta, C);
        }
        if (prec != DCSD_PREC_FP64) {
            GemmPlan p;
            std::string e;
            if (plan_einsum(spec, A, Bm, C, p, e) && p.NB == 1 && p.K >= 16)
                return einsum_tc(c, spec, alpha, A, Bm, beta, C, nsplit);
            return einsum32(c, spec, alpha, A, Bm, beta, C);
        }
        return einsum64(c, spec, alpha, A, Bm, beta, C);
    };

    // the A->B amplitude: its fixed value (fixed-reference methods), or the
    // C-condition (2D methods; zero in the CAS case)
    if (method_fr(method)) DCSD_TRY(set_fixed_amplitude(c, ref, method_fr_value(method)));
    else DCSD_TRY(apply_c_condition(c, ref));
    // t2 is final: the tensor-core operand packs of t2 views copy from its
    // BF16 image (dropped on every return)
    struct ImageScope {
        Ctx* c;
        ~ImageScope() { c->t2img_src = nullptr; }
    } image_scope{c};
    if (prec != DCSD_PREC_FP64) DCSD_TRY(t2_image(c, nsplit));

    TV B = view(c->B, {X, n, n});
    TV Bov = sub(sub(B, 1, 0, O), 2, nc, V);
    TV Bvv = sub(sub(B, 1, nc, V), 2, nc, V);
    TV t1 = view(c->t1, {2, O, V});
    TV t2 = view(c->t2, {3, O, O, V, V});
    TV R1 = view(c->R1, {2, O, V});
    TV R2 = view(c->R2, {3, O, O, V, V});
    const size_t nn2 = (size_t)n * n;
    // intermediates (fresh buffers while recording for the reverse sweep)
    TV Bd = view(scratch(c, c->Bd, 2 * X * nn2), {2, X, n, n});
    TV Z = view(scratch(c, c->Z, 2 * X * O * V), {2, X, O, V});
    TV J = view(c->J, {O, O, V, V});
    TV fd = view(scratch(c, c->fd, 2 * nn2), {2, n, n});
    auto BdVO = [&](int s) { return sub(sub(blk(Bd, s), 1, nc, V), 2, 0, O); };  // [L][a][i]
    auto BdOO = [&](int s) { return sub(sub(blk(Bd, s), 1, 0, O), 2, 0, O); };  // [L][k][i]
    auto BdVV = [&](int s) { return sub(sub(blk(Bd, s), 1, nc, V), 2, nc, V); };  // [L][a][c]
    const double* fock_s[2] = {c->fock[ref == 0 ? 0 : 1], c->fock[ref == 0 ? 1 : 0]};

    // ---- T1 dressing of the DF factors -----------------------------------
    for (int s = 0; s < 2; ++s) {
        TV t1s = blk(t1, s);
        TV P = view(scratch(c, c->Pbt, X * n * O), {X, n, O});
        DCSD_TRY(sml("Lpa,ka->Lpk", 1.0, sub(B, 2, nc, V), t1s, 0.0, P));
        TV Bds = blk(Bd, s);
        DCSD_TRY(copy_dev(c, Bds.p, c->B, X * nn2));
        DCSD_TRY(axpy_view(c, 1.0, P, 1.0, sub(Bds, 2, 0, O)));
        DCSD_TRY(sml("ka,Lkq->Laq", -1.0, t1s, sub(B, 1, 0, O), 1.0, sub(Bds, 1, nc, V)));
        DCSD_TRY(sml("ka,Lkm->Lam", -1.0, t1s, sub(P, 1, 0, O), 1.0, sub(sub(Bds, 1, nc, V), 2, 0, O)));
    }

    // ---- dressed Fock matrices -------------------------------------------
    {
        TV jv = view(scratch(c, c->fsc + 7 * nn2, X), {X});
        TV Bova = sub(sub(B, 1, 0, O), 2, nc, V);
        DCSD_TRY(sml("Lka,ka->L", 1.0, Bova, blk(t1, 0), 0.0, jv));
        DCSD_TRY(sml("Lka,ka->L", 1.0, Bova, blk(t1, 1), 1.0, jv));
        TV Jt = view(scratch(c, c->fsc, nn2), {n, n});
        DCSD_TRY(sml("Lpq,L->pq", 1.0, B, jv, 0.0, Jt));
        for (int s = 0; s < 2; ++s) {
            TV F1 = view(scratch(c, c->fsc + 1 * nn2, nn2), {n, n});
            DCSD_TRY(copy_dev(c, F1.p, fock_s[s], nn2));
            DCSD_TRY(axpy_view(c, 1.0, view(c->Kref[ref][s], {n, n}), 1.0, F1));
            DCSD_TRY(axpy_view(c, 1.0, Jt, 1.0, F1));
            TV S = view(scratch(c, c->fsc + 2 * nn2, nn2), {n, n});
            TV Tm = view(scratch(c, c->fsc + 3 * nn2, nn2), {n, n});
            DCSD_TRY(build_tau_mats(c, s, S.p, Tm.p));
            TV tmp = view(scratch(c, c->fsc + 4 * nn2, nn2), {n, n});
            DCSD_TRY(sml("pr,rq->pq", 1.0, F1, Tm, 0.0, tmp));
            TV fds = blk(fd, s);
            DCSD_TRY(sml("pr,rq->pq", 1.0, S, tmp, 0.0, fds));
            TV Bds = blk(Bd, s);
            if (nc > 0)
                DCSD_TRY(sml("Lpk,Lkq->pq", -1.0, sub(Bds, 2, 0, nc), sub(Bds, 1, 0, nc), 1.0, fds));
            DCSD_TRY(sml("Lp,Lq->pq", -1.0, fix(Bds, 2, fr.occ_act[s]), fix(Bds, 1, fr.occ_act[s]), 1.0,
                         fds));
        }
    }

    // ---- Z^s_L[i][a] = sum_{kc} T^{s.}[(ia),(kc)] B_L[k][c] ------------------
    DCSD_TRY(big("ikac,Lkc->Lia", 1.0, blk(t2, 0), Bov, 0.0, blk(Z, 0)));
    DCSD_TRY(big("ikac,Lkc->Lia", 1.0, blk(t2, 2), Bov, 1.0, blk(Z, 0)));
    DCSD_TRY(big("ikac,Lkc->Lia", 1.0, blk(t2, 1), Bov, 0.0, blk(Z, 1)));
    DCSD_TRY(big("kica,Lkc->Lia", 1.0, blk(t2, 2), Bov, 1.0, blk(Z, 1)));

    DCSD_TRY(zero_dev(c, c->R2, 3 * O * O * V * V));
    // tensor-core modes: accumulate the tensor-core contributions to R2 in FP32
    struct R2fGuard {
        Ctx* c;
        ~R2fGuard() { c->r2f_on = false; }
    } r2f_guard{c};
    if (fast) {
        if (!c->r2f) {
            if (cudaMalloc((void**)&c->r2f, sizeof(float) * 3 * O * O * V * V) != cudaSuccess) {
                cudaGetLastError();
                c->r2f = nullptr;
                c->err = "cudaMalloc of the FP32 residual accumulator failed";
                return DCSD_ERR_OOM;
            }
        }
        DCSD_CUDA(c, cudaMemsetAsync(c->r2f, 0, sizeof(float) * 3 * O * O * V * V, c->stream));
        c->r2f_on = true;
    }
    const int s1_of[3] = {0, 1, 0}, s2_of[3] = {0, 1, 1};

    // ---- <ab||ij> (dressed) -------------------------------------------------
    for (int b = 0; b < 3; ++b) {
        int s1 = s1_of[b], s2 = s2_of[b];
        DCSD_TRY(big("Lai,Lbj->ijab", 1.0, BdVO(s1), BdVO(s2), 1.0, blk(R2, b)));
        if (s1 == s2) DCSD_TRY(big("Laj,Lbi->ijab", -1.0, BdVO(s1), BdVO(s1), 1.0, blk(R2, b)));
    }

    // ---- Fock terms incl. the Fock-like quadratic terms ---------------------
    TV Foc = view(scratch(c, c->Foc, 2 * O * O), {2, O, O});
    TV Fvi = view(scratch(c, c->Fvi, 2 * V * V), {2, V, V});
    for (int s = 0; s < 2; ++s) {
        TV fds = blk(fd, s);
        DCSD_TRY(sml("Lme,Lje->mj", y, Bov, blk(Z, s), 0.0, blk(Foc, s)));
        DCSD_TRY(axpy_view(c, 1.0, sub(sub(fds, 0, 0, O), 1, 0, O), 1.0, blk(Foc, s)));
        DCSD_TRY(sml("Lme,Lmb->be", -y, Bov, blk(Z, s), 0.0, blk(Fvi, s)));
        DCSD_TRY(axpy_view(c, 1.0, sub(sub(fds, 0, nc, V), 1, nc, V), 1.0, blk(Fvi, s)));
    }
    for (int b = 0; b < 3; ++b) {
        int s1 = s1_of[b], s2 = s2_of[b];
        DCSD_TRY(big("bc,ijac->ijab", 1.0, blk(Fvi, s2), blk(t2, b), 1.0, blk(R2, b)));
        DCSD_TRY(big("ac,ijcb->ijab", 1.0, blk(Fvi, s1), blk(t2, b), 1.0, blk(R2, b)));
    }

    // ---- particle-particle ladder (undressed (ac|bd), stacked blocks) --------
    TV G = view(scratch(c, c->G, 4 * O * O * O * V), {4, O, O, O, V});
    TV H = view(scratch(c, c->H, 3 * O * O * O * O), {3, O, O, O, O});
    if (prec != DCSD_PREC_FP64) {
        // tensor cores: the fused ladder (integral tiles built on chip) with the
        // G intermediate; while recording, the tape gets the chunked ladder and
        // G-pass entries whose integrals the reverse sweep rebuilds
        const bool rec = c->rec;
        if (rec) {
            const long ch = std::max<long>(1, std::min<long>(V, (long)(c->big_elems / (V * V * V))));
            const long kc = std::max<long>(1, std::min<long>(O, (long)(c->big_elems / (V * V * V))));
            DCSD_TRY(ladder64(c, t2, Bvv, R2, c->big0, ch, nsplit, false));
            DCSD_TRY(gpass(c, t2, Bov, Bvv, G, c->big0, kc, nsplit, false));
            c->rec = false;
        }
        const dcsd_status st = ladder_tc(c, nsplit, c->R2, G.p);
        c->rec = rec;
        DCSD_TRY(st);
    } else {
        // FP64: chunked einsums (while recording, one tape entry each), or,
        // with stored four-index integrals, one contraction with them (the
        // reverse mode records the factorised form, equal to the threshold
        // of the factorisation)
        const long ch = std::max<long>(1, std::min<long>(V, (long)(c->big_elems / (V * V * V))));
        if (c->vvvv && !c->rec)
            DCSD_TRY(einsum64(c, "sijcd,acbd->sijab", 1.0, t2, view(c->vvvv, {V, V, V, V}), 1.0, R2));
        else
            DCSD_TRY(ladder64(c, t2, Bvv, R2, c->big0, ch, 0));
        // T1 corrections: G[s][ij][k][b] = sum_cd (kc|bd) t_s[ij][cd]; G[3] with
        // t_ab transposed in (c,d); H[s][ij][k][m] = sum_cd (kc|md) t_s[ij][cd]
        const long kc = std::max<long>(1, std::min<long>(O, (long)(c->big_elems / (V * V * V))));
        DCSD_TRY(gpass(c, t2, Bov, Bvv, G, c->big0, kc, 0));
    }
    DCSD_TRY(big("kmcd,sijcd->sijkm", 1.0, J, t2, 0.0, H));
    for (int b = 0; b < 3; ++b) {
        int s1 = s1_of[b], s2 = s2_of[b];
        DCSD_TRY(sml("ka,ijkb->ijab", -1.0, blk(t1, s1), blk(G, b), 1.0, blk(R2, b)));
        if (s1 == s2) DCSD_TRY(sml("mb,ijma->ijab", 1.0, blk(t1, s2), blk(G, b), 1.0, blk(R2, b)));
        else DCSD_TRY(sml("mb,ijma->ijab", -1.0, blk(t1, s2), blk(G, 3), 1.0, blk(R2, b)));
        TV tmp = view(scratch(c, c->big1, O * O * O * V), {O, O, O, V});
        DCSD_TRY(sml("ijkm,mb->ijkb", 1.0, blk(H, b), blk(t1, s2), 0.0, tmp));
        DCSD_TRY(sml("ka,ijkb->ijab", 1.0, blk(t1, s1), tmp, 1.0, blk(R2, b)));
    }

    // ---- hole-hole ladder with the quadratic ladder term --------------------
    for (int b = 0; b < 3; ++b) {
        int s1 = s1_of[b], s2 = s2_of[b];
        double cs = s1 == s2 ? 0.5 : 1.0;
        TV Wo = view(scratch(c, c->Wo, O * O * O * O), {O, O, O, O});
        DCSD_TRY(sml("Lki,Llj->klij", 1.0, BdOO(s1), BdOO(s2), 0.0, Wo));
        DCSD_TRY(axpy_view(c, cs, perm(blk(H, b), {2, 3, 0, 1}), 1.0, Wo));
        // occupied Fock terms -P(ij) sum_k F_kj t_ik^ab as part of the same
        // contraction: Wo[k][l][i][j] -= d_ki F2[l][j] + d_lj F1[k][i]
        DCSD_TRY(add_fock_hh(c, Wo.p, Foc.p + (long)s1 * O * O, Foc.p + (long)s2 * O * O));
        DCSD_TRY(big("klij,klab->ijab", 1.0, Wo, blk(t2, b), 1.0, blk(R2, b)));
    }

    // ---- ring (particle-hole) terms ------------------------------------------
    {
        TV Uex[2] = {view(scratch(c, c->big0, O * V * O * V), {O, V, O, V}),
                     view(scratch(c, c->big1, O * V * O * V), {O, V, O, V})};  // (kj|bc) as [k][c][j][b]
        for (int s = 0; s < 2; ++s) DCSD_TRY(big("Lkj,Lbc->kcjb", 1.0, BdOO(s), BdVV(s), 0.0, Uex[s]));
        TV Kq = perm(J, {0, 1, 3, 2});  // [k][l][c][d] = (kd|lc)
        auto Tm = [&](int sg, int tg) -> TV {
            if (sg == tg) return blk(t2, sg);
            if (sg == 0) return blk(t2, 2);
            return perm(blk(t2, 2), {1, 0, 3, 2});
        };
        for (int sg = 0; sg < 2; ++sg)
            for (int sp = 0; sp < 2; ++sp) {
                TV Xacc = view(scratch(c, c->big2, O * V * O * V), {O, V, O, V});
                TV Ycol = view(scratch(c, c->big3, X * O * V), {X, O, V});
                DCSD_TRY(axpy_view(c, 1.0, perm(BdVO(sp), {0, 2, 1}), 0.0, Ycol));
                DCSD_TRY(axpy_view(c, 0.5, blk(Z, sp), 1.0, Ycol));
                DCSD_TRY(big("Lia,Ljb->iajb", 1.0, blk(Z, sg), Ycol, 0.0, Xacc));
                for (int tg = 0; tg < 2; ++tg) {
                    if (tg == sp) DCSD_TRY(big("ikac,kcjb->iajb", -1.0, Tm(sg, tg), Uex[tg], 1.0, Xacc));
                    if (x != 0.0) {
                        TV scr = view(scratch(c, c->big3, O * V * O * V), {O, V, O, V});
                        DCSD_TRY(big("klcd,jlbd->kcjb", 1.0, Kq, Tm(sp, tg), 0.0, scr));
                        DCSD_TRY(big("ikac,kcjb->iajb", -0.5 * x, Tm(sg, tg), scr, 1.0, Xacc));
                    }
                }
                if (sg == sp) {
                    // R += P(ij)P(ab) X  (one pass)
                    DCSD_TRY(ring_antisym_add(c, Xacc, blk(R2, sg)));
                } else if (sg == 0) {
                    DCSD_TRY(axpy_view(c, 1.0, perm(Xacc, {0, 2, 1, 3}), 1.0, blk(R2, 2)));
                } else {
                    DCSD_TRY(add_swapped(c, Xacc, blk(R2, 2)));
                }
            }
        // mixed-spin pairs of the alpha-beta block
        TV M1 = view(scratch(c, c->big0, O * V * O * V), {O, V, O, V});  // [k][c][i][b]
        DCSD_TRY(big("Lki,Lbc->kcib", -1.0, BdOO(0), BdVV(1), 0.0, M1));
        if (x != 0.0) DCSD_TRY(big("kldc,ildb->kcib", 0.5 * x, J, blk(t2, 2), 1.0, M1));
        DCSD_TRY(big("kjac,kcib->ijab", 1.0, blk(t2, 2), M1, 1.0, blk(R2, 2)));
        TV M2 = view(scratch(c, c->big1, O * V * O * V), {O, V, O, V});  // [k][c][j][a]
        DCSD_TRY(big("Lkj,Lac->kcja", -1.0, BdOO(1), BdVV(0), 0.0, M2));
        if (x != 0.0) DCSD_TRY(big("kldc,ljad->kcja", 0.5 * x, J, blk(t2, 2), 1.0, M2));
        DCSD_TRY(big("ikcb,kcja->ijab", 1.0, blk(t2, 2), M2, 1.0, blk(R2, 2)));
    }

    // ---- singles ---------------------------------------------------------------
    for (int s = 0; s < 2; ++s) {
        TV fds = blk(fd, s);
        DCSD_TRY(axpy_view(c, 1.0, perm(sub(sub(fds, 0, nc, V), 1, 0, O), {1, 0}), 0.0, blk(R1, s)));
        DCSD_TRY(sml("Lac,Lic->ia", 1.0, BdVV(s), blk(Z, s), 1.0, blk(R1, s)));
        DCSD_TRY(sml("Lki,Lka->ia", -1.0, BdOO(s), blk(Z, s), 1.0, blk(R1, s)));
    }
    {
        auto fdOV = [&](int s) { return sub(sub(blk(fd, s), 0, 0, O), 1, nc, V); };
        DCSD_TRY(sml("kc,ikac->ia", 1.0, fdOV(0), blk(t2, 0), 1.0, blk(R1, 0)));
        DCSD_TRY(sml("kc,ikac->ia", 1.0, fdOV(1), blk(t2, 2), 1.0, blk(R1, 0)));
        DCSD_TRY(sml("kc,ikac->ia", 1.0, fdOV(1), blk(t2, 1), 1.0, blk(R1, 1)));
        DCSD_TRY(sml("kc,kica->ia", 1.0, fdOV(0), blk(t2, 2), 1.0, blk(R1, 1)));
    }

    // ---- energy Delta E_A (Eq. 2), FP64 in every precision mode ------------------
    {
        double* s = c->scal;
        for (int sp = 0; sp < 2; ++sp) {
            TV fo = sub(sub(view((double*)fock_s[sp], {n, n}), 0, 0, O), 1, nc, V);
            DCSD_TRY(dot_view(c, fo, blk(t1, sp), s + 1, sp == 0 ? 0.0 : 1.0));
        }
        for (int b = 0; b < 3; ++b) DCSD_TRY(dot_view(c, J, blk(t2, b), s + 2 + b, 0.0));
        auto ubuf = [&]() { return view(scratch(c, c->fsc + 5 * nn2, O * V), {O, V}); };
        for (int sp = 0; sp < 2; ++sp) {
            TV u = ubuf();
            DCSD_TRY(einsum64(c, "ijab,jb->ia", 1.0, J, blk(t1, sp), 0.0, u));
            DCSD_TRY(dot_view(c, u, blk(t1, sp), s + 5 + 2 * sp, 0.0));
            TV u2 = ubuf();
            DCSD_TRY(einsum64(c, "ijab,ja->ib", 1.0, J, blk(t1, sp), 0.0, u2));
            DCSD_TRY(dot_view(c, u2, blk(t1, sp), s + 6 + 2 * sp, 0.0));
        }
        TV u = ubuf();
        DCSD_TRY(einsum64(c, "ijab,jb->ia", 1.0, J, blk(t1, 1), 0.0, u));
        DCSD_TRY(dot_view(c, u, blk(t1, 0), s + 9, 0.0));
        if (c->rec) {
            TapeOp op;
            op.type = OP_ECOMB;
            rec_push(c, std::move(op));
        }
        k_energy_combine<<<1, 1, 0, c->stream>>>(s);
        DCSD_TRY(launch_check(c, "energy_combine"));
    }

    if (c->r2f_on) {
        c->r2f_on = false;
        DCSD_TRY(merge_r2f(c));
    }

    // ---- W = <B|H_N exp(T_A)|A>: R^X at the A->B double plus the products of
    // the internal singles with their residuals (zero in the CAS case);
    // two-determinant terms -------------------------------------------------------
    if (method_fr(method)) {
        const long e = (((2 * O + fr.occ_act[0]) * O + fr.occ_act[1]) * V + fr.vir_act[0]) * V + fr.vir_act[1];
        DCSD_TRY(copy_dev(c, c->scal, c->R2 + e, 1));
    } else {
        DCSD_TRY(coupling_w(c, ref));
    }
    // fixed-reference methods have no coupling terms (the element just read
    // is then the single-reference residual of the fixed excitation)
    if (method_fr(method)) DCSD_TRY(apply_fr_mask(c, ref));
    else DCSD_TRY(apply_mterms(c, ref, fast));
    return DCSD_OK;
}

}  // namespace dcsd

// Internal declarations of the 2D-CCSD/2D-DCSD residual engine (not part of
// the C ABI; see include/dcsd.h for the public interface).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dcsd.h"

namespace dcsd {

// ---------------------------------------------------------------------------
// tensor views and contraction plans
// ---------------------------------------------------------------------------
constexpr int kMaxRank = 8;
constexpr int kMaxMode = 4;

// A strided view of a dense tensor: element (i0..i_{r-1}) lives at
// p[sum_k i_k * stride[k]].  Index letters come from the einsum spec.
struct TV {
    double* p = nullptr;
    int rank = 0;
    long size[kMaxRank] = {};
    long stride[kMaxRank] = {};
};

// Build a contiguous row-major view.
TV view(double* p, std::initializer_list<long> sizes);
// Sub-view: fix/offset/slice helpers operate on a copy.
TV sub(TV v, int axis, long start, long len);   // range [start, start+len)
TV fix(TV v, int axis, long at);                // drop axis at index 'at'
TV perm(TV v, std::initializer_list<int> order);

// A contraction C[batch, m, n] = alpha * sum_k A[batch, m, k] B[batch, n, k]
// + beta * C, each of batch/m/n/k a product of up to kMaxMode strided modes.
struct GemmPlan {
    int nb = 0, nm = 0, nn = 0, nk = 0;
    long b_size[kMaxMode], b_sa[kMaxMode], b_sb[kMaxMode], b_sc[kMaxMode];
    long m_size[kMaxMode], m_sa[kMaxMode], m_sc[kMaxMode];
    long n_size[kMaxMode], n_sb[kMaxMode], n_sc[kMaxMode];
    long k_size[kMaxMode], k_sa[kMaxMode], k_sb[kMaxMode];
    long NB = 1, M = 1, N = 1, K = 1;
};

// Parse "ab,bc->ac" style specs; returns false with a message on error.
bool plan_einsum(const char* spec, const TV& A, const TV& B, const TV& C,
                 GemmPlan& plan, std::string& err);

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct MTables;   // two-determinant coupling tables (mterm.cu)
struct TcEngine;  // tensor-core contraction engine (tc_gemm.cu)

// reduction scratch (Ctx::red), in doubles
constexpr int kRedDoubles = 32768;

// ---------------------------------------------------------------------------
// reverse mode (vjp.cu): while Ctx::rec is set, the FP64 residual records
// every operation on a tape and takes fresh buffers for its intermediates
// from an arena, so that the reverse sweep sees each value as it was used.
// ---------------------------------------------------------------------------
enum TapeOpType {
    OP_EINSUM,   // C = beta C + alpha einsum(spec)(A, B)
    OP_AXPY,     // C = beta C + alpha A (strided views)
    OP_AXPY4,    // C += sum_k al[k] X[k]
    OP_COPY,     // C = A (same shape)
    OP_ZERO,     // C = 0
    OP_DOT,      // *p[0] = sum A B + beta * *p[0]
    OP_TAU,      // iarg[0] = spin: A = S = 1 - tau, B = T = 1 + tau from t1
    OP_FOCKHH,   // C = Wo -= delta F2 + delta F1 (A = F1, B = F2)
    OP_ECOMB,    // dE_A from the energy pieces in scal[1..9]
    OP_SWAPVIR,  // t2s = t2 with the virtual pair exchanged
    OP_MTERMS,   // two-determinant coupling terms, iarg[0] = ref
    OP_LADDER,   // R2 += sum_cd t2 (ac|bd), integrals rebuilt in the reverse sweep
    OP_GPASS,    // G = sum_cd t2 (kc|bd), integrals rebuilt in the reverse sweep
    OP_CCOND,    // t2[e] = -t1[p] t1[q] (C-condition; iarg: e, p, q as longs in p[])
    OP_WFULL     // W = R2[e] + t1[p] R1[q] + t1[q] R1[p] (R1 values saved in scal[50..51])
};

struct TapeOp {
    int type = 0;
    long pos[3] = {};  // OP_CCOND / OP_WFULL: element offsets e, p, q
    std::string spec;
    double alpha = 0.0, beta = 0.0;
    TV A, B, C;
    int nv = 0;
    TV X[4];
    double al[4] = {};
    int iarg[4] = {};
    double* p[4] = {};
};

struct ArenaBlock {
    double* fwd = nullptr;
    double* adj = nullptr;
    size_t cap = 0, used = 0;
};

// forward buffer and its adjoint (same element offsets)
struct AdjRegion {
    const double* fwd = nullptr;
    size_t len = 0;
    double* adj = nullptr;
};

struct Ctx {
    int nc = 0, nv = 0, X = 0;
    int n = 0, O = 0, V = 0;      // n = nc+2+nv; union occ O = nc+2; union vir V = nv+2
    int o = 0, v = 0;             // per-spin ABI sizes
    cudaStream_t stream = nullptr;
    std::string err;
    long long launches = 0;
    int device = 0;
    int num_sms = 0;

    // inputs (device, FP64)
    double* B = nullptr;          // [X][n][n]
    double* fock[2] = {};         // Phi_A alpha / beta Fock [n][n]
    double* Kref[2][2] = {};      // [ref][spin] exchange of the frame's occupied set [n][n]

    // working tensors (device, FP64), union layout
    double* t1 = nullptr;         // [2][O][V]
    double* t2 = nullptr;         // [3][O][O][V][V] (aa, bb, ab)
    double* t2s = nullptr;        // t2 with the two virtual indices exchanged (coupling terms)
    double* R1 = nullptr;         // [2][O][V]
    double* R2 = nullptr;         // [3][O][O][V][V]
    double* Bd = nullptr;         // [2][X][n][n] T1-dressed DF factors
    double* Pbt = nullptr;        // [X][n][O] scratch for dressing
    double* fd = nullptr;         // [2][n][n] dressed Fock
    double* fsc = nullptr;        // [8][n][n] small-matrix scratch
    double* Z = nullptr;          // [2][X][O][V]
    double* J = nullptr;          // [O][O][V][V] (kc|ld) (input-only, built at init)
    double* H = nullptr;          // [3][O][O][O][O]
    double* G = nullptr;          // [4][O][O][O][V] ladder T1 correction
    double* Wo = nullptr;         // [O][O][O][O]
    double* Foc = nullptr;        // [2][O][O]
    double* Fvi = nullptr;        // [2][V][V]
    double* big0 = nullptr;       // scratch >= max(ring matrices, ladder chunks)
    double* big1 = nullptr;
    double* big2 = nullptr;
    double* big3 = nullptr;
    size_t big_elems = 0;
    double* abi[10] = {};         // device staging of ABI arrays for host mem_kind calls
    double* red = nullptr;        // reduction scratch
    double* splitk_ws = nullptr;  // split-K partial tiles of the FP64 contraction kernel
    size_t splitk_elems = 0;
    double* scal = nullptr;       // device scalars: [0]=W [1]=dEA [2..] misc
    double* c1 = nullptr;         // [2][O][V] two-determinant coefficients
    // tensor-core modes: FP32 accumulator shadowing R2.  While r2f_on, the
    // tensor-core GEMMs that accumulate into R2 (beta = 1) add into r2f
    // instead (same element offsets); the residual adds it to R2 before W is
    // read.
    float* r2f = nullptr;
    bool r2f_on = false;
    // operands the tensor-core engine may keep packed between contractions
    // (pack_cache_set; valid only while their data does not change)
    const double* pack_cache_src[2] = {};
    // BF16 image of t2 for the operand packs of one tensor-core residual:
    // plane p holds part p of the split of every element (plane stride
    // t2img_plane elements).  Valid while t2img_src is set: residual_union
    // builds it after the last write to t2 and clears it on return.
    uint16_t* t2img = nullptr;
    size_t t2img_cap = 0;             // elements, all planes
    const double* t2img_src = nullptr;
    long t2img_len = 0, t2img_plane = 0;
    int t2img_planes = 0;
    double* hostbuf = nullptr;    // pinned host staging for scalars
    int ladder_chunk = 8;         // virtual rows per V build chunk (FP64)
    // the ladder contraction in clusters of two CTAs sharing each B tile by
    // TMA multicast (DCSD_TC_MULTICAST=0 selects the one-CTA kernel)
    bool tc_multicast = true;
    // operand packs: the tiled FP64 kernel only, without the t2 image and the
    // row kernel (DCSD_PACK_GENERIC=1; both give identical operands)
    bool pack_generic = false;
    // tensor-core ladder in symmetric / antisymmetric form over the (c <= d)
    // pairs (DCSD_LADDER_SA=0 selects the contraction over all (c, d))
    bool ladder_sa = true;

    MTables* mt[2] = {};          // per reference
    TcEngine* tc = nullptr;

    // optional device-time accounting (dcsd_profile)
    bool prof_on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[8];
    size_t prof_used[8] = {};
    int ladder_phase = 0;         // set while the ladder GEMMs run (profile class)
    // DCSD_TRACE=1: per-call device time by label, summarised to stderr on destroy
    bool trace = false;
    bool trace_seq = false;  // also list every tensor-core GEMM launch in order
    int tc_seq = 0;          // tensor-core GEMM launches so far
    int pack_seq = 0;        // operand pack launches so far
    bool verbose = false;         // DCSD_VERBOSE=1: per-iteration solver log on stderr
    std::string cur_spec;
    std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> trace_ev;

    // reverse mode
    bool rec = false;
    std::vector<TapeOp> tape;
    std::vector<ArenaBlock> arena;
    std::vector<AdjRegion> regions;
    double* vbuf = nullptr;       // adjoint buffers of the inputs and outputs (vjp.cu)
    size_t vbuf_elems = 0;
    double* pairbuf = nullptr;    // pair-row stacks of the tensor-core ladder reverse (vjp.cu)
    size_t pairbuf_elems = 0;

    // solver state (device)
    double* diis_t = nullptr;     // [nd][len]
    double* diis_e = nullptr;     // [nd][len]
    int diis_cap = 0;
    double* jac_s = nullptr;      // [len] Jacobi step and new amplitudes when no DIIS history is kept
    double* jac_t = nullptr;
    double* defect = nullptr;     // [len] MIXED solve: defect e = R_X6(T) - R64(T) of the last outer step
    // stored four-index integrals (ac|bd) of the union virtuals, [a][c][b][d]
    // (contexts made from FCIDUMP with the stored-integral ladder); the FP64
    // residual then takes its particle-particle ladder from them
    double* vvvv = nullptr;
};

// ---------------------------------------------------------------------------
// FP64 <-> FP32 conversion on the integer units.  On this GPU a hardware
// F64<->F32 conversion issues on the FP64 pipe, which runs at about 1/30 of
// the FP32 rate; these do the same conversion with 32-bit integer
// operations, from the IEEE 754 binary32/binary64 encodings (sign, biased
// exponent, fraction; biases 127 and 1023).  Results whose binary32 form is
// subnormal take the hardware conversion (rare: |x| < 2^-126).
// ---------------------------------------------------------------------------
// binary32 -> binary64, exact
__device__ __forceinline__ double f32_to_f64(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu, sgn = u & 0x80000000u;
    if (e == 0u) return m == 0u ? __hiloint2double((int)sgn, 0) : (double)x;
    const unsigned ed = e == 0xFFu ? 0x7FFu : e + 896u;  // 1023 - 127
    return __hiloint2double((int)(sgn | (ed << 20) | (m >> 3)), (int)(m << 29));
}

// binary64 -> binary32, round to nearest, ties to even
__device__ __forceinline__ float f64_to_f32(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sgn = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    if (e == 0x7FF) {  // infinity or NaN
        const bool nan = ((hi & 0xFFFFFu) | lo) != 0u;
        return __uint_as_float(sgn | 0x7F800000u | (nan ? 0x400000u : 0u));
    }
    const int ef = e - 896;
    if (ef >= 0xFF) return __uint_as_float(sgn | 0x7F800000u);  // overflow
    if (ef <= 0) return e == 0 ? __uint_as_float(sgn) : (float)x;  // zero / subnormal result
    const unsigned m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29), rem = lo & 0x1FFFFFFFu;
    unsigned bits = sgn | ((unsigned)ef << 23) | m23;
    if (rem > 0x10000000u || (rem == 0x10000000u && (m23 & 1u))) ++bits;  // carry may reach infinity
    return __uint_as_float(bits);
}

// error helpers
#define DCSD_CUDA(ctx, call)                                                  \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_);  \
            return DCSD_ERR_CUDA;                                             \
        }                                                                     \
    } while (0)

#define DCSD_TRY(call)                                                        \
    do {                                                                      \
        dcsd_status s_ = (call);                                              \
        if (s_ != DCSD_OK) return s_;                                         \
    } while (0)

// ---------------------------------------------------------------------------
// kernels (launchers return DCSD_OK or set ctx->err)
// ---------------------------------------------------------------------------
dcsd_status einsum64(Ctx* c, const char* spec, double alpha, const TV& A,
                     const TV& B, double beta, const TV& C);
// same contraction with FP32 products (FP64 accumulation across k-tiles);
// rows or columns of length 1 still take the FP64 matrix-vector kernel
dcsd_status einsum32(Ctx* c, const char* spec, double alpha, const TV& A,
                     const TV& B, double beta, const TV& C);
// C (+)= alpha * A elementwise over identical index sets (4D max), any strides
dcsd_status axpy_view(Ctx* c, double alpha, const TV& A, double beta, const TV& C);
// sum_i A_i * B_i over identical shapes -> *out (device pointer), FP64
dcsd_status dot_view(Ctx* c, const TV& A, const TV& B, double* out, double accumulate);
dcsd_status fill(Ctx* c, double* p, size_t n, double val);
// C += sum_k alpha_k A_k over up to 4 rank-4 views (one pass)
dcsd_status axpy4(Ctx* c, int nv, const double* alpha, const TV* A, const TV& C);
// R[i][j][a][b] += X[i][a][j][b] - X[j][a][i][b] - X[i][b][j][a] + X[j][b][i][a]
// (X [O][V][O][V], R [O][O][V][V]); recorded as that four-view axpy4
dcsd_status ring_antisym_add(Ctx* c, const TV& X, const TV& R);
// R[i][j][a][b] += X[j][b][i][a]; recorded as that axpy_view
dcsd_status add_swapped(Ctx* c, const TV& X, const TV& R);
// out[k] = <x, ys[k]> for k < m <= 16, contiguous vectors of length n (device out)
dcsd_status multidot(Ctx* c, const double* x, const double* const* ys_host, int m, long n, double* out);

// layout conversion between the ABI and the union layout
dcsd_status unpack_T(Ctx* c, int ref, const double* T1a, const double* T1b,
                     const double* T2aa, const double* T2bb, const double* T2ab);
dcsd_status pack_R(Ctx* c, int ref, double* R1a, double* R1b, double* R2aa,
                   double* R2bb, double* R2ab);
dcsd_status pack_T(Ctx* c, int ref, double* T1a, double* T1b, double* T2aa,
                   double* T2bb, double* T2ab);
dcsd_status build_tau_mats(Ctx* c, int spin, double* Smat, double* Tmat);
dcsd_status check_finite(Ctx* c, const double* p, size_t n, double* flag);

// two-determinant layer
dcsd_status mtables_build(Ctx* c);
void mtables_free(Ctx* c);
// R2 += r2f (FP32 accumulator of the tensor-core GEMMs)
dcsd_status merge_r2f(Ctx* c);
// coupling terms; fp32 = evaluate the doubles coefficient products in FP32
dcsd_status apply_mterms(Ctx* c, int ref, bool fp32);
// fixed-reference methods: zero the non-amplitude positions and the fixed
// A->B element of the residual; set the fixed amplitude in c->t2
dcsd_status apply_fr_mask(Ctx* c, int ref);
// offsets in the union layout of the two internal singles (t alpha -> u
// alpha, u beta -> t beta in frame A; their flips in frame B) in t1 / R1,
// and of the A->B doubles element in t2 / R2
struct InternalPos {
    long s1, s2, e;
};
inline InternalPos internal_pos(const Ctx* c, int ref);
// C-condition t2[A->B] = -t1[s1] t1[s2] (intermediate normalisation of the
// two-determinant wave operator; zero in the CAS case)
dcsd_status apply_c_condition(Ctx* c, int ref);
// W = R2[A->B] + t1[s1] R1[s2] + t1[s2] R1[s1] into scal[0]
dcsd_status coupling_w(Ctx* c, int ref);
dcsd_status set_fixed_amplitude(Ctx* c, int ref, double value);
// method codes (dcsd_method): DC modification, fixed-reference flag, fixed value
inline bool method_valid(int m) { return m >= DCSD_CCSD && m <= DCSD_FR_DCSD_T; }
inline bool method_dc(int m) { return m == DCSD_DCSD || m == DCSD_FR_DCSD_S || m == DCSD_FR_DCSD_T; }
inline bool method_fr(int m) { return m >= DCSD_FR_CCSD_S; }
inline double method_fr_value(int m) { return m >= DCSD_FR_CCSD_T ? -1.0 : 1.0; }

// residual orchestration (residual.cu)
dcsd_status residual_union(Ctx* c, int ref, int method, int precision);
// reverse mode helpers (vjp.cu)
// buffer for an intermediate: `normal` outside recording, a fresh arena block
// (with a zeroed adjoint twin) while recording
double* scratch(Ctx* c, double* normal, size_t elems);
void rec_push(Ctx* c, TapeOp&& op);
// device copy / zero fill that the tape records
dcsd_status copy_dev(Ctx* c, double* dst, const double* src, size_t n);
dcsd_status zero_dev(Ctx* c, double* dst, size_t n);
inline bool recording(const Ctx* c) { return c->rec; }
// ladder R2 += sum_cd t2 (ac|bd) by einsum chunks over a (integrals never
// stored beyond a chunk); nsplit 0: FP64 CUDA cores, else tensor cores with
// that many operand splits.  One tape entry while recording; compute false
// writes only that entry (a caller that produces the values another way).
dcsd_status ladder64(Ctx* c, const TV& t2, const TV& Bvv, const TV& R2, double* chunkbuf, long chunk,
                     int nsplit = 0, bool compute = true);
// ladder T1-correction intermediate G[s][ij][k][b] = sum_cd t_s[ij][cd] (kc|bd)
// (G[3] with t_ab exchanged in (c,d)) by chunks over k; one tape entry
dcsd_status gpass(Ctx* c, const TV& t2, const TV& Bov, const TV& Bvv, const TV& G, double* chunkbuf, long chunk,
                  int nsplit = 0, bool compute = true);
void vjp_free(Ctx* c);
// reverse mode in stages: record the FP64 residual at c->t1/c->t2, then any
// number of reverse sweeps with union-layout seeds; the gradients of the
// last sweep are at vjp_t1bar/vjp_t2bar (union layout) and vjp_fbar
dcsd_status vjp_record(Ctx* c, int ref, int method, int prec);
dcsd_status vjp_sweep(Ctx* c, const double* R1bar_u, const double* R2bar_u, double Ebar, double Wbar);
double* vjp_t1bar(Ctx* c);
double* vjp_t2bar(Ctx* c);
double* vjp_fbar(Ctx* c, int spin);
// adjoints of the coupling terms and of t2s (mterm.cu); pointers are the
// adjoint buffers of t1, t2, t2s, c1, R1, R2 and the scalars
dcsd_status mterms_adjoint(Ctx* c, int ref, double* t1b, double* t2b, double* t2sb, double* c1b, double* R1b,
                           double* R2b, double* scalb);
dcsd_status swap_vir_adjoint(Ctx* c, const double* t2sb, double* t2b);
// ABI <-> union amplitude layout for explicit union buffers (dir 0: ABI ->
// union, the caller zeroes the union buffers first; dir 1: union -> ABI)
dcsd_status layout_union(Ctx* c, int ref, int dir, double* u1, double* u2, double* const* abi);
dcsd_status add_fock_hh(Ctx* c, double* Wo, const double* F1, const double* F2);
// J = (kc|ld) and the reference exchange matrices K_ref from B.  While
// recording it writes only the tape entries (the context already holds these
// products of the unchanged B); prec selects the engine of J's adjoint.
dcsd_status init_constants(Ctx* c, int prec = DCSD_PREC_FP64);
// one OP_EINSUM tape entry (engine 0 FP64, 1 FP32, 2 tensor cores with nsplit)
void record_einsum(Ctx* c, const char* spec, double alpha, const TV& A, const TV& B, double beta, const TV& C,
                   int engine, int nsplit);

// tensor-core engine (tc_gemm.cu)
dcsd_status tc_init(Ctx* c);
void tc_free(Ctx* c);
// same contract as einsum64 with BF16 (nsplit=1) or split BF16 (nsplit=2,
// three products) operands on tcgen05 tensor cores, FP32 accumulation
dcsd_status einsum_tc(Ctx* c, const char* spec, double alpha, const TV& A,
                      const TV& B, double beta, const TV& C, int nsplit);

// pp ladder + its T1 correction on tensor cores (R2 += ladder, G = correction)
dcsd_status ladder_tc(Ctx* c, int nsplit, double* R2, double* G);
// sources whose packed operands einsum_tc may reuse (NULL: none); clears the cache
void pack_cache_set(Ctx* c, const double* src0, const double* src1);
// the BF16 image of t2 with the parts of an nsplit-way split (see Ctx)
dcsd_status t2_image(Ctx* c, int nsplit);

// record a CUDA event pair around a launch of class cls when profiling
inline void prof_begin(Ctx* c, int cls) {
    if (!c->prof_on) return;
    auto& v = c->prof_ev[cls];
    if (c->prof_used[cls] == v.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        v.push_back({a, b});
    }
    cudaEventRecord(v[c->prof_used[cls]].first, c->stream);
}
inline void prof_end(Ctx* c, int cls) {
    if (!c->prof_on) return;
    cudaEventRecord(c->prof_ev[cls][c->prof_used[cls]].second, c->stream);
    c->prof_used[cls]++;
}

inline void trace_begin(Ctx* c, const std::string& label) {
    if (!c->trace) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, c->stream);
    c->trace_ev.push_back({label, {a, b}});
}
inline void trace_end(Ctx* c) {
    if (!c->trace || c->trace_ev.empty()) return;
    cudaEventRecord(c->trace_ev.back().second.second, c->stream);
}
void trace_report(Ctx* c);

inline dcsd_status launch_check(Ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string(what) + ": " + cudaGetErrorString(e);
        return DCSD_ERR_CUDA;
    }
    c->launches++;
    return DCSD_OK;
}

// frame description (which union positions are valid for each spin)
struct Frame {
    int occ_act[2];   // union occ index of the active occupied orbital per spin
    int vir_act[2];   // union vir index of the active virtual orbital per spin
};
inline Frame frame_of(const Ctx* c, int ref) {
    Frame f;
    int t = c->nc, u = c->nc + 1;
    if (ref == 0) {
        f.occ_act[0] = t; f.occ_act[1] = u; f.vir_act[0] = 1; f.vir_act[1] = 0;
    } else {
        f.occ_act[0] = u; f.occ_act[1] = t; f.vir_act[0] = 0; f.vir_act[1] = 1;
    }
    return f;
}
inline InternalPos internal_pos(const Ctx* c, int ref) {
    const Frame f = frame_of(c, ref);
    const long O = c->O, V = c->V;
    InternalPos p;
    p.s1 = (0 * O + f.occ_act[0]) * V + f.vir_act[0];
    p.s2 = (1 * O + f.occ_act[1]) * V + f.vir_act[1];
    p.e = (((2 * O + f.occ_act[0]) * O + f.occ_act[1]) * V + f.vir_act[0]) * V + f.vir_act[1];
    return p;
}

}  // namespace dcsd

struct dcsd_ctx {
    dcsd::Ctx c;
};

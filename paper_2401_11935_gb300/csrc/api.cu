// C ABI entry points (include/dcsd.h): context management, residual/energy
// calls, the on-device Jacobi + DIIS solver and the 2x2 effective
// Hamiltonian of the two references (arXiv 2401.11935, Section II).
#include "common.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

using namespace dcsd;

static std::string g_init_error;

namespace dcsd {

// Jacobi step on the concatenated union vector [t1 (2*O*V) | t2 (3*O*O*V*V)]:
// step = -R / D with D the Fock-diagonal orbital-energy differences of the
// frame (zero where R is zero: padding, masked and symmetry-forbidden
// elements); tnew = t + step.
// 1/D for the Jacobi step: FP32 reciprocal refined by one Newton-Raphson
// iteration r <- r (2 - D r) in FP64 (relative error about 2^-46), a few FP64
// operations instead of a full-precision division
__device__ __forceinline__ double recip_nr(double D) {
    double r = (double)__frcp_rn((float)D);
    return fma(r, fma(-D, r, 1.0), r);
}

// Jacobi step on the concatenated amplitude vector: one block per row --
// 2*O rows of T1 (length V), then 3*O*O rows of T2 (length V*V).  The
// virtual diagonal Fock elements of the row's spins are staged in shared
// memory (2*V doubles of dynamic shared memory, or read from the Fock
// matrices when stage is false).
// F32: the doubles' step -R/D is formed in FP32 (tensor-core precisions;
// the step only has to be a good preconditioned direction, the update
// t + step and the stored vectors stay FP64)
template <bool F32>
__global__ void __launch_bounds__(256) k_jacobi_rows(int n, int nc, int O, int V, const double* fa,
                                                     const double* fb, const double* t, const double* R,
                                                     double* tnew, double* step, bool stage) {
    extern __shared__ double jdiag[];  // [2][V]
    const long nrow1 = 2l * O, nrow = nrow1 + 3l * O * O;
    for (long row = blockIdx.x; row < nrow; row += gridDim.x) {
        int blk, i, j;
        if (row < nrow1) {
            blk = (int)(row / O);  // spin of the T1 row
            i = (int)(row % O);
            j = -1;
        } else {
            const long r2 = row - nrow1;
            blk = (int)(r2 / ((long)O * O));
            i = (int)((r2 / O) % O);
            j = (int)(r2 % O);
        }
        const bool is1 = j < 0;
        const double* f1 = is1 ? (blk == 0 ? fa : fb) : (blk == 1 ? fb : fa);
        const double* f2 = is1 ? f1 : (blk == 0 ? fa : fb);
        const double* d1 = f1 + (long)nc * n + nc;  // diagonal, stride n + 1
        const double* d2 = f2 + (long)nc * n + nc;
        long d1s = n + 1, d2s = n + 1;
        if (stage) {
            __syncthreads();  // previous row done with the staged diagonal
            for (int x = threadIdx.x; x < V; x += blockDim.x) {
                jdiag[x] = d1[(long)x * (n + 1)];
                jdiag[V + x] = d2[(long)x * (n + 1)];
            }
            __syncthreads();
            d1 = jdiag;
            d2 = jdiag + V;
            d1s = d2s = 1;
        }
        if (is1) {
            const long base = row * V;
            const double dij = f1[(long)i * n + i];
            for (int x = threadIdx.x; x < V; x += blockDim.x) {
                const double r = R[base + x];
                const double st = r != 0.0 ? -r * recip_nr(d1[x * d1s] - dij) : 0.0;
                step[base + x] = st;
                tnew[base + x] = t[base + x] + st;
            }
        } else {
            const long base = 2l * O * V + (row - nrow1) * V * V;
            const double dij = f1[(long)i * n + i] + f2[(long)j * n + j];
            const unsigned VV = (unsigned)V * (unsigned)V, bs = blockDim.x;
            // four elements per thread and pass (eight loads in flight)
            for (unsigned e0 = threadIdx.x; e0 < VV; e0 += 4 * bs) {
                double r[4], tt[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const unsigned e = e0 + q * bs;
                    r[q] = e < VV ? R[base + e] : 0.0;
                    tt[q] = e < VV ? t[base + e] : 0.0;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const unsigned e = e0 + q * bs;
                    if (e >= VV) break;
                    const unsigned x = e / (unsigned)V, b = e - x * (unsigned)V;
                    double st;
                    if (F32) {
                        const float rf = f64_to_f32(r[q]);
                        const float Df = f64_to_f32(d1[x * d1s] - dij) + f64_to_f32(d2[b * d2s]);
                        st = rf != 0.0f ? f32_to_f64(-rf * __frcp_rn(Df)) : 0.0;
                    } else {
                        st = r[q] != 0.0 ? -r[q] * recip_nr(d1[x * d1s] - dij + d2[b * d2s]) : 0.0;
                    }
                    step[base + e] = st;
                    tnew[base + e] = tt[q] + st;
                }
            }
        }
    }
}

// max |p[e]| per block; with flag set, a non-finite element also sets
// *flag = 1 (one pass for the convergence measure and the finiteness check).
// The max runs on the integer units: with the sign bit cleared, the bit
// patterns of finite doubles order as their magnitudes, and every Inf or NaN
// pattern lies above them (exponent all ones), which is the flag's test.
__global__ void k_maxabs_partial(const double* p, long n, double* part, double* flag) {
    __shared__ unsigned long long sh[256];
    const unsigned long long* q = (const unsigned long long*)p;
    const unsigned long long mask = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long m = 0;
    const long stride = (long)gridDim.x * blockDim.x;
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    for (; e + 3 * stride < n; e += 4 * stride) {
        const unsigned long long x0 = q[e] & mask, x1 = q[e + stride] & mask, x2 = q[e + 2 * stride] & mask,
                                 x3 = q[e + 3 * stride] & mask;
        m = max(max(m, x0), max(x1, max(x2, x3)));
    }
    for (; e < n; e += stride) m = max(m, q[e] & mask);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = max(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (flag && sh[0] >= 0x7FF0000000000000ull) *flag = 1.0;
        part[blockIdx.x] = __longlong_as_double((long long)sh[0]);
    }
}

__global__ void k_maxabs_final(const double* part, int n, double* out) {
    __shared__ double sh[256];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) m = fmax(m, part[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

struct LinComb {
    const double* v[16];
    double coef[16];
    int m;
};

__global__ void __launch_bounds__(256) k_lincomb(LinComb lc, long n, double* out) {
    const long stride = (long)gridDim.x * blockDim.x;
    long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
    for (; e + stride < n; e += 2 * stride) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < lc.m; ++k) {
            s0 += lc.coef[k] * lc.v[k][e];
            s1 += lc.coef[k] * lc.v[k][e + stride];
        }
        out[e] = s0;
        out[e + stride] = s1;
    }
    if (e < n) {
        double s0 = 0.0;
        for (int k = 0; k < lc.m; ++k) s0 += lc.coef[k] * lc.v[k][e];
        out[e] = s0;
    }
}

static unsigned grid_n(Ctx* c, long n) {
    long g = (n + 255) / 256, cap = (long)std::max(c->num_sms, 1) * 8;
    return (unsigned)std::max<long>(1, std::min(g, cap));
}

static dcsd_status maxabs(Ctx* c, const double* p, long n, double* out, double* flag = nullptr) {
    k_maxabs_partial<<<512, 256, 0, c->stream>>>(p, n, c->red, flag);
    DCSD_TRY(launch_check(c, "maxabs_partial"));
    k_maxabs_final<<<1, 256, 0, c->stream>>>(c->red, 512, out);
    return launch_check(c, "maxabs_final");
}

}  // namespace dcsd

// ---------------------------------------------------------------------------
namespace {

struct AbiBufs {
    double* p[5] = {};
};

long abi_len(const Ctx* c, int k) {
    return k < 2 ? (long)c->o * c->v : (long)c->o * c->o * c->v * c->v;
}

dcsd_status alloc(Ctx* c, double** p, size_t n) {
    if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "cudaMalloc of " + std::to_string(n * sizeof(double)) + " bytes failed";
        return DCSD_ERR_OOM;
    }
    return DCSD_OK;
}

void free_ctx(Ctx* c) {
    double** ptrs[] = {&c->B, &c->fock[0], &c->fock[1], &c->Kref[0][0], &c->Kref[0][1],
                       &c->Kref[1][0], &c->Kref[1][1], &c->t1, &c->R1, &c->t2s, &c->Bd, &c->Pbt, &c->fd,
                       &c->fsc, &c->Z, &c->J, &c->H, &c->G, &c->Wo, &c->Foc, &c->Fvi, &c->big0,
                       &c->big1, &c->big2, &c->big3, &c->red, &c->splitk_ws, &c->scal, &c->c1, &c->diis_t,
                       &c->diis_e, &c->jac_s, &c->jac_t, &c->defect, &c->abi[0], &c->abi[1], &c->abi[2], &c->abi[3], &c->abi[4],
                       &c->abi[5], &c->abi[6], &c->abi[7], &c->abi[8], &c->abi[9]};
    for (auto pp : ptrs) {
        if (*pp) cudaFree(*pp);
        *pp = nullptr;
    }
    c->t2 = nullptr;
    c->R2 = nullptr;
    if (c->vvvv) cudaFree(c->vvvv);
    c->vvvv = nullptr;
    if (c->r2f) cudaFree(c->r2f);
    c->r2f = nullptr;
    if (c->t2img) cudaFree(c->t2img);
    c->t2img = nullptr;
    c->t2img_cap = 0;
    c->t2img_src = nullptr;
    if (c->hostbuf) cudaFreeHost(c->hostbuf);
    c->hostbuf = nullptr;
    for (int k = 0; k < 8; ++k) {
        for (auto& e : c->prof_ev[k]) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        c->prof_ev[k].clear();
    }
    mtables_free(c);
    tc_free(c);
    vjp_free(c);
}

// device ABI staging (host mem_kind)
dcsd_status ensure_abi(Ctx* c) {
    if (c->abi[0]) return DCSD_OK;
    for (int k = 0; k < 10; ++k) DCSD_TRY(alloc(c, &c->abi[k], abi_len(c, k % 5)));
    return DCSD_OK;
}

// DIIS history of nd vectors of length len (grow-only, kept until destroy)
dcsd_status ensure_diis(Ctx* c, int nd, long len) {
    if (nd <= c->diis_cap) return DCSD_OK;
    if (c->diis_t) cudaFree(c->diis_t);
    if (c->diis_e) cudaFree(c->diis_e);
    c->diis_t = c->diis_e = nullptr;
    c->diis_cap = 0;
    DCSD_TRY(alloc(c, &c->diis_t, (size_t)nd * len));
    DCSD_TRY(alloc(c, &c->diis_e, (size_t)nd * len));
    c->diis_cap = nd;
    return DCSD_OK;
}

// step / new-amplitude vectors of a Jacobi-only solve (kept until destroy)
dcsd_status ensure_jacobi(Ctx* c, long len) {
    if (!c->jac_s) DCSD_TRY(alloc(c, &c->jac_s, len));
    if (!c->jac_t) DCSD_TRY(alloc(c, &c->jac_t, len));
    return DCSD_OK;
}

dcsd_status sync_scalars(Ctx* c, int count) {
    DCSD_CUDA(c, cudaMemcpyAsync(c->hostbuf, c->scal, sizeof(double) * count, cudaMemcpyDeviceToHost,
                                 c->stream));
    DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
    return DCSD_OK;
}

// the tensor-core kernels record a bounded-wait expiry in scal[22] (int)
bool tc_timeout(Ctx* c) {
    int flag;
    std::memcpy(&flag, &c->hostbuf[22], sizeof(int));
    if (flag != 0) {
        c->err = "tensor-core pipeline wait expired (code " + std::to_string(flag) + ")";
        return true;
    }
    return false;
}

bool valid_prec(int p) {
    return p == DCSD_PREC_FP64 || p == DCSD_PREC_BF16 || p == DCSD_PREC_BF16X3 || p == DCSD_PREC_BF16X6;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" dcsd_status dcsd_init(dcsd_ctx** out, const dcsd_dims* d, const double* eps,
                                 const double* fock_a, const double* fock_b, const double* B,
                                 int mem_kind, void* stream) {
    (void)eps;
    if (!out) {
        g_init_error = "out is NULL";
        return DCSD_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!d || !fock_a || !fock_b || !B) {
        g_init_error = "NULL argument";
        return DCSD_ERR_INVALID_ARG;
    }
    if (d->n_c < 0 || d->n_v < 1 || d->naux < 1 || (mem_kind != DCSD_MEM_HOST && mem_kind != DCSD_MEM_DEVICE)) {
        g_init_error = "invalid dimensions or mem_kind";
        return DCSD_ERR_INVALID_ARG;
    }
    int dev = 0, ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_init_error = "no CUDA device";
        return DCSD_ERR_NO_DEVICE;
    }
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    if (prop.major != 10 || prop.minor != 3) {
        g_init_error = "device is sm_" + std::to_string(prop.major) + std::to_string(prop.minor) +
                       "; this library is built for sm_103a (GB300)";
        return DCSD_ERR_NO_DEVICE;
    }
    dcsd_ctx* h = new dcsd_ctx();
    Ctx* c = &h->c;
    c->device = dev;
    c->num_sms = prop.multiProcessorCount;
    c->stream = (cudaStream_t)stream;
    {
        const char* tr = getenv("DCSD_TRACE");
        c->trace = tr && (tr[0] == '1' || tr[0] == '2');
        c->trace_seq = tr && tr[0] == '2';
        const char* vb = getenv("DCSD_VERBOSE");
        c->verbose = vb && vb[0] == '1';
        const char* mc = getenv("DCSD_TC_MULTICAST");
        c->tc_multicast = !(mc && mc[0] == '0');
        const char* pg = getenv("DCSD_PACK_GENERIC");
        c->pack_generic = pg && pg[0] == '1';
        const char* ls = getenv("DCSD_LADDER_SA");
        c->ladder_sa = !(ls && ls[0] == '0');
    }
    c->nc = d->n_c;
    c->nv = d->n_v;
    c->X = d->naux;
    c->n = c->nc + 2 + c->nv;
    c->O = c->nc + 2;
    c->V = c->nv + 2;
    c->o = c->nc + 1;
    c->v = c->nv + 1;
    const size_t n = c->n, O = c->O, V = c->V, X = c->X;
    const size_t OV = O * V, n1 = 2 * OV, n2 = 3 * OV * OV;
    c->big_elems = std::max({OV * OV, V * V * V, X * OV, O * O * O * V, (size_t)16});
    auto fail = [&](dcsd_status s) {
        g_init_error = c->err;
        free_ctx(c);
        delete h;
        return s;
    };
    dcsd_status st = DCSD_OK;
#define A_(p, cnt) if ((st = alloc(c, &(p), (cnt))) != DCSD_OK) return fail(st)
    A_(c->B, X * n * n);
    A_(c->fock[0], n * n);
    A_(c->fock[1], n * n);
    for (int r = 0; r < 2; ++r)
        for (int s = 0; s < 2; ++s) A_(c->Kref[r][s], n * n);
    A_(c->t1, n1 + n2);
    c->t2 = c->t1 + n1;
    A_(c->R1, n1 + n2);
    c->R2 = c->R1 + n1;
    A_(c->c1, n1);
    A_(c->t2s, n2);
    A_(c->Bd, 2 * X * n * n);
    A_(c->Pbt, X * n * O);
    A_(c->fd, 2 * n * n);
    A_(c->fsc, 7 * n * n + X + 16);
    A_(c->Z, 2 * X * OV);
    A_(c->J, OV * OV);
    A_(c->H, 3 * O * O * O * O);
    A_(c->G, 4 * O * O * O * V);
    A_(c->Wo, O * O * O * O);
    A_(c->Foc, 2 * O * O);
    A_(c->Fvi, 2 * V * V);
    A_(c->big0, c->big_elems);
    A_(c->big1, c->big_elems);
    A_(c->big2, c->big_elems);
    A_(c->big3, c->big_elems);
    A_(c->red, kRedDoubles);
    c->splitk_elems = std::max<size_t>(1 << 20, std::min<size_t>(64ul << 20, 16 * (n * n + O * V)));
    A_(c->splitk_ws, c->splitk_elems);
    A_(c->scal, 64);
#undef A_
    if (cudaMallocHost((void**)&c->hostbuf, 64 * sizeof(double)) != cudaSuccess) {
        c->err = "cudaMallocHost failed";
        return fail(DCSD_ERR_OOM);
    }
    cudaMemcpyKind kind = mem_kind == DCSD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(c->B, B, X * n * n * sizeof(double), kind, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->fock[0], fock_a, n * n * sizeof(double), kind, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->fock[1], fock_b, n * n * sizeof(double), kind, c->stream) != cudaSuccess) {
        c->err = std::string("input copy failed: ") + cudaGetErrorString(cudaGetLastError());
        return fail(DCSD_ERR_CUDA);
    }
    if ((st = init_constants(c)) != DCSD_OK) return fail(st);
    if ((st = mtables_build(c)) != DCSD_OK) return fail(st);
    if ((st = tc_init(c)) != DCSD_OK) return fail(st);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        c->err = std::string("init: ") + cudaGetErrorString(cudaGetLastError());
        return fail(DCSD_ERR_CUDA);
    }
    *out = h;
    return DCSD_OK;
}

extern "C" dcsd_status dcsd_destroy(dcsd_ctx* h) {
    if (!h) return DCSD_OK;
    Ctx* c = &h->c;
    cudaStreamSynchronize(c->stream);
    trace_report(c);
    free_ctx(c);
    delete h;
    return DCSD_OK;
}

extern "C" const char* dcsd_last_error(const dcsd_ctx* h) {
    if (!h) return g_init_error.c_str();
    return h->c.err.c_str();
}

extern "C" long long dcsd_kernel_launches(const dcsd_ctx* h) { return h ? h->c.launches : 0; }

extern "C" dcsd_status dcsd_profile(dcsd_ctx* h, int enable, int reset, double* ms, long long* launches) {
    if (!h) return DCSD_ERR_INVALID_ARG;
    Ctx* c = &h->c;
    if (ms || launches) {
        DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int k = 0; k < DCSD_PROF_NCLASS; ++k) {
            double sum = 0.0;
            for (size_t i = 0; i < c->prof_used[k]; ++i) {
                float t = 0.f;
                DCSD_CUDA(c, cudaEventElapsedTime(&t, c->prof_ev[k][i].first, c->prof_ev[k][i].second));
                sum += t;
            }
            if (ms) ms[k] = sum;
            if (launches) launches[k] = (long long)c->prof_used[k];
        }
    }
    if (reset)
        for (int k = 0; k < DCSD_PROF_NCLASS; ++k) c->prof_used[k] = 0;
    c->prof_on = enable != 0;
    return DCSD_OK;
}

static dcsd_status residual_common(Ctx* c, int ref, int method, int prec, int mem_kind,
                                   const double* const* T, double* const* R, double* W, double* dEA) {
    if ((ref != 0 && ref != 1) || !method_valid(method) || !valid_prec(prec) ||
        (mem_kind != DCSD_MEM_HOST && mem_kind != DCSD_MEM_DEVICE)) {
        c->err = "invalid ref/method/precision/mem_kind";
        return DCSD_ERR_INVALID_ARG;
    }
    for (int k = 0; k < 5; ++k)
        if (!T[k]) {
            c->err = "NULL amplitude pointer";
            return DCSD_ERR_INVALID_ARG;
        }
    const double* Td[5];
    double* Rd[5] = {};
    if (mem_kind == DCSD_MEM_HOST) {
        DCSD_TRY(ensure_abi(c));
        for (int k = 0; k < 5; ++k) {
            DCSD_CUDA(c, cudaMemcpyAsync(c->abi[k], T[k], abi_len(c, k) * sizeof(double),
                                         cudaMemcpyHostToDevice, c->stream));
            Td[k] = c->abi[k];
            Rd[k] = c->abi[5 + k];
        }
    } else {
        for (int k = 0; k < 5; ++k) {
            Td[k] = T[k];
            Rd[k] = R ? R[k] : nullptr;
        }
    }
    DCSD_TRY(unpack_T(c, ref, Td[0], Td[1], Td[2], Td[3], Td[4]));
    DCSD_TRY(residual_union(c, ref, method, prec));
    if (R) {
        for (int k = 0; k < 5; ++k)
            if (!R[k]) {
                c->err = "NULL residual pointer";
                return DCSD_ERR_INVALID_ARG;
            }
        DCSD_TRY(pack_R(c, ref, Rd[0], Rd[1], Rd[2], Rd[3], Rd[4]));
    }
    DCSD_CUDA(c, cudaMemsetAsync(c->scal + 20, 0, sizeof(double), c->stream));
    DCSD_TRY(check_finite(c, c->R1, 2ul * c->O * c->V + 3ul * c->O * c->O * c->V * c->V, c->scal + 20));
    if (mem_kind == DCSD_MEM_HOST && R) {
        for (int k = 0; k < 5; ++k)
            DCSD_CUDA(c, cudaMemcpyAsync(R[k], Rd[k], abi_len(c, k) * sizeof(double), cudaMemcpyDeviceToHost,
                                         c->stream));
    }
    DCSD_TRY(sync_scalars(c, 23));
    if (tc_timeout(c)) return DCSD_ERR_TIMEOUT;
    if (W) *W = c->hostbuf[0];
    if (dEA) *dEA = c->hostbuf[1];
    if (c->hostbuf[20] != 0.0 || !std::isfinite(c->hostbuf[0]) || !std::isfinite(c->hostbuf[1])) {
        c->err = "non-finite residual";
        return DCSD_ERR_NUMERIC;
    }
    return DCSD_OK;
}

extern "C" dcsd_status dcsd_residual(dcsd_ctx* h, int ref, int method, int precision, int mem_kind,
                                     const double* T1a, const double* T1b, const double* T2aa,
                                     const double* T2bb, const double* T2ab, double* R1a, double* R1b,
                                     double* R2aa, double* R2bb, double* R2ab, double* W, double* dEA) {
    if (!h) return DCSD_ERR_INVALID_ARG;
    Ctx* c = &h->c;
    const double* T[5] = {T1a, T1b, T2aa, T2bb, T2ab};
    double* R[5] = {R1a, R1b, R2aa, R2bb, R2ab};
    for (int k = 0; k < 5; ++k)
        if (!R[k]) {
            c->err = "NULL residual pointer";
            return DCSD_ERR_INVALID_ARG;
        }
    return residual_common(c, ref, method, precision, mem_kind, T, R, W, dEA);
}

extern "C" dcsd_status dcsd_energy(dcsd_ctx* h, int ref, int method, int mem_kind, const double* T1a,
                                   const double* T1b, const double* T2aa, const double* T2bb,
                                   const double* T2ab, double* dEA, double* W) {
    if (!h) return DCSD_ERR_INVALID_ARG;
    const double* T[5] = {T1a, T1b, T2aa, T2bb, T2ab};
    return residual_common(&h->c, ref, method, DCSD_PREC_FP64, mem_kind, T, nullptr, W, dEA);
}

// Reservation: every buffer a residual of the given precision (and a solve
// with diis_n history vectors, and host-memory staging) touches is allocated
// now.  The buffers of the tensor-core engine are sized by the contractions
// that use them and only ever grow, and their sizes depend on the dimensions
// alone, so one residual at zero amplitudes through the same code path sizes
// every one of them (CCSD's term set contains every contraction of DCSD).
extern "C" dcsd_status dcsd_reserve(dcsd_ctx* h, int precision, int diis_n, int host_staging) {
    if (!h) return DCSD_ERR_INVALID_ARG;
    Ctx* c = &h->c;
    if ((!valid_prec(precision) && precision != DCSD_PREC_MIXED) || diis_n < 0 || diis_n > 16 ||
        (host_staging != 0 && host_staging != 1)) {
        c->err = "dcsd_reserve: invalid precision, diis_n or host_staging";
        return DCSD_ERR_INVALID_ARG;
    }
    const long len = 2l * c->O * c->V + 3l * c->O * c->O * c->V * c->V;
    if (host_staging) DCSD_TRY(ensure_abi(c));
    if (diis_n > 0) DCSD_TRY(ensure_diis(c, diis_n, len));
    else DCSD_TRY(ensure_jacobi(c, len));
    int runs[2] = {-1, -1};
    if (precision == DCSD_PREC_MIXED) {
        runs[0] = DCSD_PREC_BF16;
        runs[1] = DCSD_PREC_BF16X6;
        if (!c->defect) DCSD_TRY(alloc(c, &c->defect, len));
    } else if (precision != DCSD_PREC_FP64) {
        runs[0] = precision;
    }
    for (int r : runs) {
        if (r < 0) continue;
        DCSD_CUDA(c, cudaMemsetAsync(c->t1, 0, len * sizeof(double), c->stream));
        DCSD_TRY(residual_union(c, 0, DCSD_CCSD, r));
    }
    DCSD_TRY(sync_scalars(c, 23));
    if (tc_timeout(c)) return DCSD_ERR_TIMEOUT;
    return DCSD_OK;
}

namespace dcsd {
dcsd_status vjp_run(Ctx* c, int ref, int method, int prec, const double* const* Td, const double* const* Rb,
                    double Ebar, double Wbar, double* const* Tb, double* Bb, double* Fab, double* Fbb);
}

extern "C" dcsd_status dcsd_vjp(dcsd_ctx* h, int ref, int method, int precision, int mem_kind, const double* T1a,
                                const double* T1b, const double* T2aa, const double* T2bb, const double* T2ab,
                                const double* R1a_bar, const double* R1b_bar, const double* R2aa_bar,
                                const double* R2bb_bar, const double* R2ab_bar, double dEA_bar, double W_bar,
                                double* T1a_bar, double* T1b_bar, double* T2aa_bar, double* T2bb_bar,
                                double* T2ab_bar, double* B_bar, double* fock_a_bar, double* fock_b_bar) {
    if (!h) return DCSD_ERR_INVALID_ARG;
    Ctx* c = &h->c;
    const double* T[5] = {T1a, T1b, T2aa, T2bb, T2ab};
    const double* Rb[5] = {R1a_bar, R1b_bar, R2aa_bar, R2bb_bar, R2ab_bar};
    double* Tb[5] = {T1a_bar, T1b_bar, T2aa_bar, T2bb_bar, T2ab_bar};
    // reverse mode: the 2D methods (the fixed-reference residual has a fixed
    // amplitude, whose derivative the recorded tape does not exclude)
    if ((ref != 0 && ref != 1) || (method != DCSD_CCSD && method != DCSD_DCSD) || !valid_prec(precision) ||
        (mem_kind != DCSD_MEM_HOST && mem_kind != DCSD_MEM_DEVICE)) {
        c->err = "invalid ref/method/precision/mem_kind";
        return DCSD_ERR_INVALID_ARG;
    }
    int nrb = 0;
    for (int k = 0; k < 5; ++k) {
        if (!T[k] || !Tb[k]) {
            c->err = "NULL amplitude or amplitude-gradient pointer";
            return DCSD_ERR_INVALID_ARG;
        }
        nrb += Rb[k] != nullptr;
    }
    if (nrb != 0 && nrb != 5) {
        c->err = "residual cotangents must be all NULL or all given";
        return DCSD_ERR_INVALID_ARG;
    }
    const size_t nn = (size_t)c->n * c->n, nB = (size_t)c->X * nn;
    if (mem_kind == DCSD_MEM_DEVICE)
        return vjp_run(c, ref, method, precision, T, nrb ? Rb : nullptr, dEA_bar, W_bar, Tb, B_bar, fock_a_bar,
                       fock_b_bar);
    // host memory: stage through device buffers
    DCSD_TRY(ensure_abi(c));
    std::vector<double*> tmp;
    struct Free {
        std::vector<double*>& v;
        ~Free() { for (double* p : v) cudaFree(p); }
    } fr{tmp};
    auto dev = [&](size_t n) -> double* {
        double* p = nullptr;
        if (alloc(c, &p, n) != DCSD_OK) return nullptr;
        tmp.push_back(p);
        return p;
    };
    const double* Td[5];
    const double* Rd[5] = {};
    double* Tbd[5];
    for (int k = 0; k < 5; ++k) {
        const size_t len = abi_len(c, k);
        DCSD_CUDA(c, cudaMemcpyAsync(c->abi[k], T[k], len * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        Td[k] = c->abi[k];
        if (nrb) {
            DCSD_CUDA(c, cudaMemcpyAsync(c->abi[5 + k], Rb[k], len * sizeof(double), cudaMemcpyHostToDevice,
                                         c->stream));
            Rd[k] = c->abi[5 + k];
        }
        if (!(Tbd[k] = dev(len))) return DCSD_ERR_OOM;
    }
    double* Bd = nullptr;
    double* Fad = nullptr;
    double* Fbd = nullptr;
    if (B_bar && !(Bd = dev(nB))) return DCSD_ERR_OOM;
    if (fock_a_bar && !(Fad = dev(nn))) return DCSD_ERR_OOM;
    if (fock_b_bar && !(Fbd = dev(nn))) return DCSD_ERR_OOM;
    DCSD_TRY(vjp_run(c, ref, method, precision, Td, nrb ? Rd : nullptr, dEA_bar, W_bar, Tbd, Bd, Fad, Fbd));
    for (int k = 0; k < 5; ++k)
        DCSD_CUDA(c, cudaMemcpyAsync(Tb[k], Tbd[k], abi_len(c, k) * sizeof(double), cudaMemcpyDeviceToHost,
                                     c->stream));
    if (Bd) DCSD_CUDA(c, cudaMemcpyAsync(B_bar, Bd, nB * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (Fad) DCSD_CUDA(c, cudaMemcpyAsync(fock_a_bar, Fad, nn * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (Fbd) DCSD_CUDA(c, cudaMemcpyAsync(fock_b_bar, Fbd, nn * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
    return DCSD_OK;
}

// small dense solve (partial pivoting) of the DIIS system
static bool solve_small(int m, std::vector<double> A, std::vector<double> b, std::vector<double>& x) {
    for (int k = 0; k < m; ++k) {
        int piv = k;
        for (int i = k + 1; i < m; ++i)
            if (std::fabs(A[i * m + k]) > std::fabs(A[piv * m + k])) piv = i;
        if (std::fabs(A[piv * m + k]) < 1e-300) return false;
        if (piv != k) {
            for (int j = 0; j < m; ++j) std::swap(A[k * m + j], A[piv * m + j]);
            std::swap(b[k], b[piv]);
        }
        for (int i = k + 1; i < m; ++i) {
            double f = A[i * m + k] / A[k * m + k];
            for (int j = k; j < m; ++j) A[i * m + j] -= f * A[k * m + j];
            b[i] -= f * b[k];
        }
    }
    x.assign(m, 0.0);
    for (int i = m - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < m; ++j) s -= A[i * m + j] * x[j];
        x[i] = s / A[i * m + i];
    }
    return true;
}

namespace {

// same-spin blocks (0, 1) of a union [3][O][O][V][V] array projected onto
// arrays antisymmetric in (i,j) and in (a,b)
__global__ void k_antisym_ss(long O, long V, double* x) {
    const long total = 2 * O * O * V * V;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long blk = e / (O * O * V * V), r = e - blk * O * O * V * V;
        const long i = r / (O * V * V), j = (r / (V * V)) % O, a = (r / V) % V, b = r % V;
        if (i > j || a > b) continue;  // one thread per quadruple
        double* X = x + blk * O * O * V * V;
        auto at = [&](long p, long q, long c, long d) -> double& { return X[((p * O + q) * V + c) * V + d]; };
        if (i == j || a == b) {
            at(i, j, a, b) = at(j, i, a, b) = at(i, j, b, a) = at(j, i, b, a) = 0.0;
            continue;
        }
        const double v = 0.25 * (at(i, j, a, b) - at(j, i, a, b) - at(i, j, b, a) + at(j, i, b, a));
        at(i, j, a, b) = v;
        at(j, i, a, b) = -v;
        at(i, j, b, a) = -v;
        at(j, i, b, a) = v;
    }
}

}  // namespace

// Lambda equations of the Lagrangian L = E(T) + sum_q Lambda_q R_q(T) with
// E = dE_A + state * W (state +1 singlet, -1 triplet), at converged T:
//     dL/dT = dE/dT + Lambda^T dR/dT = 0,
// solved by Jacobi steps with the amplitude denominators and DIIS; every
// iteration is one reverse sweep of the recorded FP64 residual with seeds
// (Lambda, 1, state).  The response density gamma^sigma_pq = dL/df^sigma_pq
// is the Fock-matrix gradient of the final sweep.
extern "C" dcsd_status dcsd_lambda(dcsd_ctx* h, const dcsd_solve_opts* o, int state, int mem_kind,
                                   const double* T1a, const double* T1b, const double* T2aa, const double* T2bb,
                                   const double* T2ab, double* L1a, double* L1b, double* L2aa, double* L2bb,
                                   double* L2ab, double* rdm_a, double* rdm_b, dcsd_result* res) {
    if (!h || !o || !res) return DCSD_ERR_INVALID_ARG;
    Ctx* c = &h->c;
    const double* T[5] = {T1a, T1b, T2aa, T2bb, T2ab};
    double* Lio[5] = {L1a, L1b, L2aa, L2bb, L2ab};
    if ((o->ref != 0 && o->ref != 1) || (o->method != DCSD_CCSD && o->method != DCSD_DCSD) ||
        o->precision != DCSD_PREC_FP64 || o->maxiter < 1 || o->diis_n < 0 || o->diis_n > 16 || !(o->tol > 0.0) ||
        (state != 1 && state != -1) || (mem_kind != DCSD_MEM_HOST && mem_kind != DCSD_MEM_DEVICE)) {
        c->err = "invalid Lambda options (precision must be FP64, state +1 or -1)";
        return DCSD_ERR_INVALID_ARG;
    }
    for (int k = 0; k < 5; ++k)
        if (!T[k] || !Lio[k]) {
            c->err = "NULL amplitude or Lambda pointer";
            return DCSD_ERR_INVALID_ARG;
        }
    auto t0 = std::chrono::steady_clock::now();
    const int ref = o->ref;
    const long n1 = 2l * c->O * c->V, len = n1 + 3l * c->O * c->O * c->V * c->V;
    const size_t nn = (size_t)c->n * c->n;
    std::vector<double*> tmp;
    struct Free {
        std::vector<double*>& v;
        ~Free() { for (double* p : v) cudaFree(p); }
    } fr{tmp};
    auto dev = [&](size_t n) -> double* {
        double* p = nullptr;
        if (alloc(c, &p, n) != DCSD_OK) return nullptr;
        tmp.push_back(p);
        return p;
    };
    // amplitudes and Lambda guess on the device (ABI layout)
    const double* Td[5];
    double* Ld[5];
    for (int k = 0; k < 5; ++k) {
        const size_t l = abi_len(c, k);
        if (mem_kind == DCSD_MEM_HOST) {
            double* p = dev(l);
            double* q = dev(l);
            if (!p || !q) return DCSD_ERR_OOM;
            DCSD_CUDA(c, cudaMemcpyAsync(p, T[k], l * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            if (o->use_guess)
                DCSD_CUDA(c, cudaMemcpyAsync(q, Lio[k], l * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            Td[k] = p;
            Ld[k] = q;
        } else {
            Td[k] = T[k];
            Ld[k] = Lio[k];
        }
    }
    double* lam = dev(len);   // union Lambda [t1-like | t2-like]
    double* gp = dev(len);    // projected gradient
    double* abt[5];           // ABI staging for the projection
    for (int k = 0; k < 5; ++k)
        if (!(abt[k] = dev(abi_len(c, k)))) return DCSD_ERR_OOM;
    if (!lam || !gp) return DCSD_ERR_OOM;
    DCSD_CUDA(c, cudaMemsetAsync(lam, 0, len * sizeof(double), c->stream));
    if (o->use_guess) DCSD_TRY(layout_union(c, ref, 0, lam, lam + n1, Ld));
    // record the residual at T
    DCSD_TRY(unpack_T(c, ref, Td[0], Td[1], Td[2], Td[3], Td[4]));
    DCSD_TRY(vjp_record(c, ref, o->method, DCSD_PREC_FP64));
    struct TapeClear {
        Ctx* c;
        ~TapeClear() { c->tape.clear(); }
    } tc_guard{c};
    DCSD_TRY(sync_scalars(c, 2));
    res->W = c->hostbuf[0];
    res->dEA = c->hostbuf[1];
    res->E_S = res->dEA + res->W;
    res->E_T = res->dEA - res->W;
    res->switched_at = -1;
    res->polished_at = -1;
    res->converged = 0;
    const Frame frm = frame_of(c, ref);
    const long eAB = n1 + (((2l * c->O + frm.occ_act[0]) * c->O + frm.occ_act[1]) * c->V + frm.vir_act[0]) * c->V +
                     frm.vir_act[1];
    const int nd = o->diis_n;
    if (nd > 0) DCSD_TRY(ensure_diis(c, nd, len));
    double* sbuf = nd == 0 ? dev(len) : nullptr;
    double* tbuf = nd == 0 ? dev(len) : nullptr;
    if (nd == 0 && (!sbuf || !tbuf)) return DCSD_ERR_OOM;
    const double* fa = c->fock[ref == 0 ? 0 : 1];
    const double* fb = c->fock[ref == 0 ? 1 : 0];
    std::vector<double> Bm(16 * 16, 0.0);
    int nhist = 0, next = 0, it = 0;
    dcsd_status status = DCSD_ERR_NOT_CONVERGED;
    for (it = 1; it <= o->maxiter; ++it) {
        DCSD_CUDA(c, cudaMemsetAsync(lam + eAB, 0, sizeof(double), c->stream));
        DCSD_TRY(vjp_sweep(c, lam, lam + n1, 1.0, (double)state));
        // gradient in the independent parameters: valid positions only, the
        // same-spin doubles antisymmetric, the A->B double fixed
        DCSD_TRY(layout_union(c, ref, 1, vjp_t1bar(c), vjp_t2bar(c), abt));
        DCSD_CUDA(c, cudaMemsetAsync(gp, 0, len * sizeof(double), c->stream));
        DCSD_TRY(layout_union(c, ref, 0, gp, gp + n1, abt));
        k_antisym_ss<<<grid_n(c, 2l * c->O * c->O * c->V * c->V), 256, 0, c->stream>>>(c->O, c->V, gp + n1);
        DCSD_TRY(launch_check(c, "antisym_ss"));
        DCSD_CUDA(c, cudaMemsetAsync(gp + eAB, 0, sizeof(double), c->stream));
        DCSD_TRY(maxabs(c, gp, len, c->scal + 21));
        DCSD_TRY(sync_scalars(c, 22));
        const double gmax = c->hostbuf[21];
        res->max_r = gmax;
        if (c->verbose) fprintf(stderr, "[dcsd lambda] it %3d max|G| %.3e\n", it, gmax);
        if (!std::isfinite(gmax)) {
            c->err = "non-finite Lambda gradient";
            status = DCSD_ERR_NUMERIC;
            break;
        }
        if (gmax <= o->tol) {
            status = DCSD_OK;
            res->converged = 1;
            break;
        }
        double* st_v = nd > 0 ? c->diis_e + (size_t)next * len : sbuf;
        double* tn_v = nd > 0 ? c->diis_t + (size_t)next * len : tbuf;
        {
            const size_t jsm = 2ul * c->V * sizeof(double);
            const bool stage = jsm <= 48 * 1024;
            const unsigned jg = (unsigned)std::min<long>(2l * c->O + 3l * c->O * c->O, (long)c->num_sms * 8);
            k_jacobi_rows<false><<<jg, 256, stage ? jsm : 0, c->stream>>>(c->n, c->nc, c->O, c->V, fa, fb, lam,
                                                                           gp, tn_v, st_v, stage);
            DCSD_TRY(launch_check(c, "lambda_jacobi"));
        }
        if (nd == 0) {
            DCSD_CUDA(c, cudaMemcpyAsync(lam, tn_v, len * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            continue;
        }
        const int cur = next;
        next = (next + 1) % nd;
        nhist = std::min(nhist + 1, nd);
        {
            const double* ys[16];
            for (int j = 0; j < nhist; ++j) ys[j] = c->diis_e + (size_t)((cur - j + nd) % nd) * len;
            DCSD_TRY(multidot(c, st_v, ys, nhist, len, c->scal + 24));
        }
        DCSD_CUDA(c, cudaMemcpyAsync(c->hostbuf + 24, c->scal + 24, sizeof(double) * nhist, cudaMemcpyDeviceToHost,
                                     c->stream));
        DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int j = 0; j < nhist; ++j) {
            const int sl = (cur - j + nd) % nd;
            Bm[cur * 16 + sl] = Bm[sl * 16 + cur] = c->hostbuf[24 + j];
        }
        LinComb lc;
        lc.m = 0;
        if (nhist >= 2) {
            const int m = nhist + 1;
            std::vector<double> A(m * m, 0.0), bb(m, 0.0), xx;
            std::vector<int> sl(nhist);
            for (int j = 0; j < nhist; ++j) sl[j] = (cur - j + nd) % nd;
            double scale = 0.0;
            for (int a = 0; a < nhist; ++a) scale = std::max(scale, std::fabs(Bm[sl[a] * 16 + sl[a]]));
            if (scale <= 0.0) scale = 1.0;
            for (int a = 0; a < nhist; ++a)
                for (int b = 0; b < nhist; ++b) A[a * m + b] = Bm[sl[a] * 16 + sl[b]] / scale;
            for (int a = 0; a < nhist; ++a) { A[a * m + nhist] = -1.0; A[nhist * m + a] = -1.0; }
            bb[nhist] = -1.0;
            if (solve_small(m, A, bb, xx))
                for (int j = 0; j < nhist; ++j) {
                    lc.v[lc.m] = c->diis_t + (size_t)sl[j] * len;
                    lc.coef[lc.m] = xx[j];
                    lc.m++;
                }
        }
        if (lc.m == 0) {
            lc.v[0] = tn_v;
            lc.coef[0] = 1.0;
            lc.m = 1;
        }
        k_lincomb<<<grid_n(c, len), 256, 0, c->stream>>>(lc, len, lam);
        DCSD_TRY(launch_check(c, "lambda_diis"));
    }
    res->iters = std::min(it, o->maxiter);
    // outputs: Lambda (ABI) and the response density of the last sweep
    DCSD_TRY(layout_union(c, ref, 1, lam, lam + n1, Ld));
    if (mem_kind == DCSD_MEM_HOST)
        for (int k = 0; k < 5; ++k)
            DCSD_CUDA(c, cudaMemcpyAsync(Lio[k], Ld[k], abi_len(c, k) * sizeof(double), cudaMemcpyDeviceToHost,
                                         c->stream));
    double* rd[2] = {rdm_a, rdm_b};
    for (int s2 = 0; s2 < 2; ++s2)
        if (rd[s2])
            DCSD_CUDA(c, cudaMemcpyAsync(rd[s2], vjp_fbar(c, s2), nn * sizeof(double),
                                         mem_kind == DCSD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                         c->stream));
    DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

extern "C" dcsd_status dcsd_heff(double dEA, double W, double* H, double* evals, int* singlet_index) {
    if (!H || !evals || !singlet_index) return DCSD_ERR_INVALID_ARG;
    H[0] = dEA; H[1] = W; H[2] = W; H[3] = dEA;
    double lo = dEA - std::fabs(W), hi = dEA + std::fabs(W);
    evals[0] = lo;
    evals[1] = hi;
    *singlet_index = W >= 0.0 ? 1 : 0;  // the singlet is dEA + W
    return DCSD_OK;
}


extern "C" dcsd_status dcsd_solve(dcsd_ctx* h, const dcsd_solve_opts* o, int mem_kind, double* T1a,
                                  double* T1b, double* T2aa, double* T2bb, double* T2ab, dcsd_result* res) {
    if (!h || !o || !res) return DCSD_ERR_INVALID_ARG;
    Ctx* c = &h->c;
    if ((o->ref != 0 && o->ref != 1) || !method_valid(o->method) ||
        (!valid_prec(o->precision) && o->precision != DCSD_PREC_MIXED) || o->maxiter < 1 ||
        o->diis_n < 0 || o->diis_n > 16 || !(o->tol > 0.0) ||
        (mem_kind != DCSD_MEM_HOST && mem_kind != DCSD_MEM_DEVICE)) {
        c->err = "invalid solve options";
        return DCSD_ERR_INVALID_ARG;
    }
    double* Tio[5] = {T1a, T1b, T2aa, T2bb, T2ab};
    for (int k = 0; k < 5; ++k)
        if (!Tio[k]) {
            c->err = "NULL amplitude pointer";
            return DCSD_ERR_INVALID_ARG;
        }
    auto t0 = std::chrono::steady_clock::now();
    const int ref = o->ref;
    const long len = 2l * c->O * c->V + 3l * c->O * c->O * c->V * c->V;
    double* Td[5];
    if (mem_kind == DCSD_MEM_HOST) {
        DCSD_TRY(ensure_abi(c));
        for (int k = 0; k < 5; ++k) Td[k] = c->abi[k];
    } else {
        for (int k = 0; k < 5; ++k) Td[k] = Tio[k];
    }
    if (o->use_guess) {
        if (mem_kind == DCSD_MEM_HOST)
            for (int k = 0; k < 5; ++k)
                DCSD_CUDA(c, cudaMemcpyAsync(Td[k], Tio[k], abi_len(c, k) * sizeof(double),
                                             cudaMemcpyHostToDevice, c->stream));
        DCSD_TRY(unpack_T(c, ref, Td[0], Td[1], Td[2], Td[3], Td[4]));
    } else {
        DCSD_CUDA(c, cudaMemsetAsync(c->t1, 0, len * sizeof(double), c->stream));
    }
    const int nd = o->diis_n;
    if (nd > 0) DCSD_TRY(ensure_diis(c, nd, len));
    else DCSD_TRY(ensure_jacobi(c, len));
    std::vector<double> Bm(16 * 16, 0.0);
    int nhist = 0, next = 0;
    // MIXED phases: 0 BF16, 1 BF16X6, 2 FP64
    int phase = 0;
    bool switched = false;
    int switched_at = -1, polished_at = -1;
    double best_r = 1e300, best_r_window = 1e300;
    int stall = 0;
    const double* fa = c->fock[ref == 0 ? 0 : 1];
    const double* fb = c->fock[ref == 0 ? 1 : 0];
    double* sbuf = c->jac_s;
    double* tbuf = c->jac_t;
    dcsd_status status = DCSD_ERR_NOT_CONVERGED;
    res->converged = 0;
    res->switched_at = -1;
    res->polished_at = -1;
    // MIXED phase 2, defect correction: an outer step evaluates the FP64
    // residual R64(T) and the BF16X6 one at the same T and keeps their
    // difference e; inner steps iterate on r(T) = R_X6(T) - e, which equals
    // R64 at the outer T and differs from R64 nearby only by the change of
    // the tensor cores' rounding error.  Convergence is declared on outer
    // (FP64) residuals only.
    bool outer = true;
    int inner = 0;
    double inner_best = 1e300;
    const TV Rall = view(c->R1, {len});
    int it = 0;
    for (it = 1; it <= o->maxiter; ++it) {
        int prec = o->precision;
        const bool refining = o->precision == DCSD_PREC_MIXED && phase == 2;
        if (prec == DCSD_PREC_MIXED)
            prec = phase == 0 ? DCSD_PREC_BF16 : phase == 1 ? DCSD_PREC_BF16X6
                                                             : (outer ? DCSD_PREC_FP64 : DCSD_PREC_BF16X6);
        dcsd_status s = residual_union(c, ref, o->method, prec);
        if (s != DCSD_OK) { status = s; break; }
        if (refining && !outer) {
            if ((s = axpy_view(c, -1.0, view(c->defect, {len}), 1.0, Rall)) != DCSD_OK) { status = s; break; }
        }
        // max|R| and the finiteness flag in one pass
        DCSD_CUDA(c, cudaMemsetAsync(c->scal + 20, 0, sizeof(double), c->stream));
        if ((s = maxabs(c, c->R1, len, c->scal + 21, c->scal + 20)) != DCSD_OK) { status = s; break; }
        if ((s = sync_scalars(c, 23)) != DCSD_OK) { status = s; break; }
        if (tc_timeout(c)) { status = DCSD_ERR_TIMEOUT; break; }
        const double W = c->hostbuf[0], dE = c->hostbuf[1], rmax = c->hostbuf[21];
        if (c->verbose)
            fprintf(stderr, "[dcsd solve] it %3d prec %d max|R| %.3e dEA %.12f W %.12f\n", it, prec, rmax, dE, W);
        res->W = W;
        res->dEA = dE;
        res->max_r = rmax;
        if (c->hostbuf[20] != 0.0 || !std::isfinite(rmax)) {
            c->err = "non-finite residual in solve";
            status = DCSD_ERR_NUMERIC;
            break;
        }
        if (rmax <= o->tol && (!refining || outer)) {
            status = DCSD_OK;
            res->converged = 1;
            break;
        }
        if (refining && outer) {
            // e = R_X6(T) - R64(T); the step below uses R64
            if (!c->defect && (s = alloc(c, &c->defect, len)) != DCSD_OK) { status = s; break; }
            double* defect = c->defect;
            DCSD_CUDA(c, cudaMemcpyAsync(defect, c->R1, len * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            if ((s = residual_union(c, ref, o->method, DCSD_PREC_BF16X6)) != DCSD_OK) { status = s; break; }
            if ((s = axpy_view(c, 1.0, Rall, -1.0, view(defect, {len}))) != DCSD_OK) { status = s; break; }
            if ((s = axpy_view(c, -1.0, view(defect, {len}), 1.0, Rall)) != DCSD_OK) { status = s; break; }
            outer = false;
            inner = 0;
            inner_best = rmax;
            nhist = 0;  // a new defect defines a new iteration function
            next = 0;
        } else if (refining) {
            // back to an outer step once the inner residual is far below the
            // target or has stopped decreasing
            ++inner;
            if (rmax < 0.5 * inner_best) { inner_best = rmax; stall = 0; }
            else ++stall;
            if (rmax <= 0.1 * o->tol || inner >= 20 || stall >= 4) {
                outer = true;
                stall = 0;
            }
        }
        // MIXED: leave BF16 once max|R| is below switch_tol or has stopped
        // decreasing (BF16 rounding puts a floor under the residual)
        if (o->precision == DCSD_PREC_MIXED && phase < 2) {
            best_r = std::min(best_r, rmax);
            if (rmax < best_r_window * 0.5) { best_r_window = rmax; stall = 0; }
            else ++stall;
            bool next_phase = false;
            if (phase == 0 && (rmax < o->switch_tol || stall >= 6)) {
                switched = true;
                switched_at = it;
                next_phase = true;
            } else if (phase == 1 && o->polish_tol > 0.0 && (rmax < o->polish_tol || stall >= 4)) {
                polished_at = it;
                next_phase = true;
            }
            if (next_phase) {
                ++phase;
                stall = 0;
                best_r_window = rmax;
                nhist = 0;  // history built with the lower precision is discarded
                next = 0;
                outer = true;
            }
        }
        double* st_v = nd > 0 ? c->diis_e + (size_t)next * len : sbuf;
        double* tn_v = nd > 0 ? c->diis_t + (size_t)next * len : tbuf;
        trace_begin(c, "jacobi");
        {
            const size_t jsm = 2ul * c->V * sizeof(double);
            const bool stage = jsm <= 48 * 1024;
            const unsigned jg = (unsigned)std::min<long>(2l * c->O + 3l * c->O * c->O, (long)c->num_sms * 8);
            if (prec != DCSD_PREC_BF16 && prec != DCSD_PREC_BF16X3)
                k_jacobi_rows<false><<<jg, 256, stage ? jsm : 0, c->stream>>>(c->n, c->nc, c->O, c->V, fa, fb,
                                                                               c->t1, c->R1, tn_v, st_v, stage);
            else
                k_jacobi_rows<true><<<jg, 256, stage ? jsm : 0, c->stream>>>(c->n, c->nc, c->O, c->V, fa, fb,
                                                                              c->t1, c->R1, tn_v, st_v, stage);
        }
        trace_end(c);
        if ((s = launch_check(c, "jacobi")) != DCSD_OK) { status = s; break; }
        if (nd == 0) {
            DCSD_CUDA(c, cudaMemcpyAsync(c->t1, tn_v, len * sizeof(double), cudaMemcpyDeviceToDevice,
                                         c->stream));
            continue;
        }
        const int cur = next;
        next = (next + 1) % nd;
        nhist = std::min(nhist + 1, nd);
        // new row of the DIIS matrix
        {
            const double* ys[16];
            for (int j = 0; j < nhist; ++j) ys[j] = c->diis_e + (size_t)((cur - j + nd) % nd) * len;
            if ((s = multidot(c, st_v, ys, nhist, len, c->scal + 24)) != DCSD_OK) { status = s; break; }
        }
        DCSD_CUDA(c, cudaMemcpyAsync(c->hostbuf + 24, c->scal + 24, sizeof(double) * nhist,
                                     cudaMemcpyDeviceToHost, c->stream));
        DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int j = 0; j < nhist; ++j) {
            int sl = (cur - j + nd) % nd;
            Bm[cur * 16 + sl] = Bm[sl * 16 + cur] = c->hostbuf[24 + j];
        }
        LinComb lc;
        lc.m = 0;
        if (nhist >= 2) {
            int m = nhist + 1;
            std::vector<double> A(m * m, 0.0), bb(m, 0.0), xx;
            std::vector<int> sl(nhist);
            for (int j = 0; j < nhist; ++j) sl[j] = (cur - j + nd) % nd;
            double scale = 0.0;
            for (int a = 0; a < nhist; ++a) scale = std::max(scale, std::fabs(Bm[sl[a] * 16 + sl[a]]));
            if (scale <= 0.0) scale = 1.0;
            for (int a = 0; a < nhist; ++a)
                for (int b = 0; b < nhist; ++b) A[a * m + b] = Bm[sl[a] * 16 + sl[b]] / scale;
            for (int a = 0; a < nhist; ++a) { A[a * m + nhist] = -1.0; A[nhist * m + a] = -1.0; }
            bb[nhist] = -1.0;
            if (solve_small(m, A, bb, xx)) {
                for (int j = 0; j < nhist; ++j) {
                    lc.v[lc.m] = c->diis_t + (size_t)sl[j] * len;
                    lc.coef[lc.m] = xx[j];
                    lc.m++;
                }
            }
        }
        if (lc.m == 0) {
            lc.v[0] = tn_v;
            lc.coef[0] = 1.0;
            lc.m = 1;
        }
        trace_begin(c, "diis_lincomb");
        k_lincomb<<<grid_n(c, len), 256, 0, c->stream>>>(lc, len, c->t1);
        trace_end(c);
        if ((s = launch_check(c, "diis_extrapolate")) != DCSD_OK) { status = s; break; }
    }
    res->iters = std::min(it, o->maxiter);
    res->E_S = res->dEA + res->W;
    res->E_T = res->dEA - res->W;
    if (method_fr(o->method)) {
        // one state: its energy is the single-reference Delta E
        const bool singlet = method_fr_value(o->method) > 0.0;
        res->E_S = singlet ? res->dEA : std::nan("");
        res->E_T = singlet ? std::nan("") : res->dEA;
    }
    res->switched_at = switched_at;
    res->polished_at = polished_at;
    // amplitudes out
    dcsd_status ps = pack_T(c, ref, Td[0], Td[1], Td[2], Td[3], Td[4]);
    if (ps != DCSD_OK) return ps;
    if (mem_kind == DCSD_MEM_HOST)
        for (int k = 0; k < 5; ++k)
            DCSD_CUDA(c, cudaMemcpyAsync(Tio[k], Td[k], abi_len(c, k) * sizeof(double), cudaMemcpyDeviceToHost,
                                         c->stream));
    DCSD_CUDA(c, cudaStreamSynchronize(c->stream));
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return status;
}

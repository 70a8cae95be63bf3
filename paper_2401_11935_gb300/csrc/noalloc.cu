// dcsd_energy_noalloc: the reference energy correlation term Delta E_A
// computed without allocating any device memory.
//
// Who needs this: code that cannot call cudaMalloc -- for example a caller
// that is recording a CUDA graph (allocation calls are not allowed inside a
// capture), a runtime whose device memory is owned by its own pool allocator,
// or an embedding that must keep a fixed memory footprint.  Such a caller
// passes only its own input and output buffers; the working memory of this
// entry point is one fixed array that is part of the loaded library.
//
// Scratch: g_energy_scratch holds one partial sum per (spin block, i, j)
// triple, i.e. 3 * o^2 doubles with o = n_c + 1; the array has room for
// kScratchDoubles, so o is limited to 52 (3 * 52^2 = 8112).  The array is
// loaded with the library and stays allocated on every device that used it
// until the process exits.  Every call writes all the slots it later reads,
// so nothing carries over from the previous call's contents, but the array
// is shared by all calls: two calls that overlap on the GPU (different
// streams, or host threads) race on it and must be serialised by the caller.
#include "common.h"

namespace {

constexpr int kScratchDoubles = 8192;
constexpr int kMaxDevices = 64;

// file-scope device scratch (the only working memory of this entry point)
static __device__ __align__(256) double g_energy_scratch[kScratchDoubles];

// host-side device address of g_energy_scratch, per device
static double* g_scratch_ptr[kMaxDevices] = {};

struct EArgs {
    int nc, o, v, n, X, ref;
    const double* fa;  // frame alpha Fock [n][n]
    const double* fb;  // frame beta Fock [n][n]
    const double* B;   // [X][n][n]
    const double* t1a;
    const double* t1b;
    const double* t2aa;
    const double* t2bb;
    const double* t2ab;
    double* partial;   // device address of g_energy_scratch
};

__device__ __forceinline__ int occ_sp(const EArgs& a, int s, int I) {
    if (I < a.nc) return I;
    // active occupied: ref 0 -> alpha t, beta u; ref 1 -> alpha u, beta t
    return a.nc + ((a.ref == 0) == (s == 0) ? 0 : 1);
}
__device__ __forceinline__ int vir_sp(const EArgs& a, int s, int A) {
    if (A > 0) return a.nc + 1 + A;
    // active virtual: ref 0 -> alpha u, beta t; ref 1 -> alpha t, beta u
    return a.nc + ((a.ref == 0) == (s == 0) ? 1 : 0);
}

// block (blk, i, j): sum_ab (ia|jb) w tau_blk[ij][ab] (+ sum_a f_ia t_ia when
// j == 0 and blk is a same-spin block of that spin); w = 1/2 for the
// same-spin blocks, 1 for alpha-beta.  (ia|jb) = sum_L B_L[ia] B_L[jb].
__global__ void k_energy_partials(EArgs a) {
    const int slot = blockIdx.x;
    const int blk = slot / (a.o * a.o), i = (slot / a.o) % a.o, j = slot % a.o;
    const int s1 = blk == 1 ? 1 : 0, s2 = blk == 0 ? 0 : 1;
    const double* t1s1 = s1 == 0 ? a.t1a : a.t1b;
    const double* t1s2 = s2 == 0 ? a.t1a : a.t1b;
    const double* t2 = blk == 0 ? a.t2aa : blk == 1 ? a.t2bb : a.t2ab;
    const long nn = (long)a.n * a.n;
    const int pi = occ_sp(a, s1, i), pj = occ_sp(a, s2, j);
    double acc = 0.0;
    for (int e = threadIdx.x; e < a.v * a.v; e += blockDim.x) {
        const int A = e / a.v, Bi = e % a.v;
        const int pa = vir_sp(a, s1, A), pb = vir_sp(a, s2, Bi);
        double J = 0.0;
        for (int L = 0; L < a.X; ++L) J = fma(a.B[L * nn + (long)pi * a.n + pa], a.B[L * nn + (long)pj * a.n + pb], J);
        double tau = t2[(((long)i * a.o + j) * a.v + A) * a.v + Bi];
        if (blk == 2) {
            tau += t1s1[i * a.v + A] * t1s2[j * a.v + Bi];
            acc = fma(J, tau, acc);
        } else {
            tau += t1s1[i * a.v + A] * t1s1[j * a.v + Bi] - t1s1[i * a.v + Bi] * t1s1[j * a.v + A];
            acc = fma(0.5 * J, tau, acc);
        }
    }
    if (blk < 2 && j == 0) {
        const double* f = blk == 0 ? a.fa : a.fb;
        for (int A = threadIdx.x; A < a.v; A += blockDim.x)
            acc = fma(f[(long)pi * a.n + vir_sp(a, s1, A)], t1s1[i * a.v + A], acc);
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.partial[slot] = sh[0];
}

// fixed-order sum of the partials (deterministic)
__global__ void k_energy_sum(const double* partial, int nslot, double* out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < nslot; k += 256) s += partial[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

extern "C" dcsd_status dcsd_energy_noalloc(int n_c, int n_v, int naux, int ref, const double* fock_a,
                                           const double* fock_b, const double* B, const double* T1a,
                                           const double* T1b, const double* T2aa, const double* T2bb,
                                           const double* T2ab, double* dEA, void* stream) {
    if (n_c < 0 || n_v < 1 || naux < 1 || (ref != 0 && ref != 1) || !fock_a || !fock_b || !B || !T1a ||
        !T1b || !T2aa || !T2bb || !T2ab || !dEA)
        return DCSD_ERR_INVALID_ARG;
    const int o = n_c + 1, v = n_v + 1;
    const long nslot = 3l * o * o;
    if (nslot > kScratchDoubles) return DCSD_ERR_INVALID_ARG;  // n_c + 1 > 52: scratch too small
    // set-up, once per device, with that device current: the device address
    // of the static scratch array (its host-side name is not that address)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return DCSD_ERR_NO_DEVICE;
    }
    if (!g_scratch_ptr[dev]) {
        double* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_energy_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DCSD_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    EArgs a;
    a.nc = n_c;
    a.o = o;
    a.v = v;
    a.n = n_c + 2 + n_v;
    a.X = naux;
    a.ref = ref;
    // the frame's alpha Fock matrix is the input beta one for ref 1 (spin flip)
    a.fa = ref == 0 ? fock_a : fock_b;
    a.fb = ref == 0 ? fock_b : fock_a;
    a.B = B;
    a.t1a = T1a;
    a.t1b = T1b;
    a.t2aa = T2aa;
    a.t2bb = T2bb;
    a.t2ab = T2ab;
    a.partial = g_scratch_ptr[dev];
    cudaStream_t st = (cudaStream_t)stream;
    k_energy_partials<<<(unsigned)nslot, 256, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return DCSD_ERR_CUDA;
    k_energy_sum<<<1, 256, 0, st>>>(g_scratch_ptr[dev], (int)nslot, dEA);
    if (cudaGetLastError() != cudaSuccess) return DCSD_ERR_CUDA;
    return DCSD_OK;
}

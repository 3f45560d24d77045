// PD local step on sm_103a, fused with the RHS assembly: per-tet deformation
// gradient, 3x3 SVD, rotation and volume targets, the per-corner
// right-hand-side contributions (in shared memory), and their deterministic
// sum per vertex into b (or into the residual b - K x).
//
// Paper: Sec. 7.1 (local step; R by polar decomposition through the SVD
// F = U Sigma W^T; V through the three-unknown problem of Eq. vol_pre with
// targets clamped to >= 0.01), Eq. pd_local, Eq. energy (per-element
// gamma_s, gamma_v).
//
// SVD: cyclic Jacobi eigen-decomposition of F^T F (Golub & Van Loan,
// "Matrix Computations", the two-sided symmetric Schur rotation), sorted
// eigenvectors W in SO(3), then a Givens QR of F W (the structure used by
// McAdams et al. 2011, "Computing the SVD of 3x3 matrices with minimal
// branching") so that U in SO(3) and the last singular value carries the
// sign of det F; a final one-sided Jacobi rotation of the trailing 2x2 block
// keeps the two smallest singular values accurate when sigma_1 / sigma_3 is
// beyond the FP32 resolution of F^T F.
//
// Volume target: minimise sum (d_i - s_i)^2 s.t. prod d = 1, d_i >= 0.01.
// KKT: (d_i - s_i) d_i = mu for the free targets.  The smallest target
// t = d_3 parameterises every candidate root: mu = t (t - s_3) and
// d_{1,2} = (s_i + sqrt(s_i^2 + 4 mu)) / 2.  On t >= s_3/2 the product is
// increasing (all roots on the + branch: safeguarded Newton); on
// [0.01, s_3/2) d_3 is the - root of its quadratic (scan and bisection of
// every sign change, only where a bound of the product allows a root).  The
// cheapest candidate is kept; the face with d_3 clamped to 0.01 (d_1 d_2 = 100,
// the same construction) is tried when the first face has no feasible point
// or a - root under the clamp; failing both, d = (1e4, 0.01, 0.01).
//
// The serving loop runs the same block code over every resident request in
// one launch (k_b_local_assemble, k_b_assemble_shared).

#include <algorithm>

#include "pd_internal.h"
#include "proj3.cuh"

namespace pdg {

namespace {

using namespace proj;

__global__ void __launch_bounds__(256) k_project(const float* __restrict__ Fin, int n, float* __restrict__ Rout,
                                                 float* __restrict__ Vout, float* __restrict__ sout) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = Fin[9 * (int64_t)e + 3 * i + j];
    float U[3][3], W[3][3], s[3], d[3], P[3][3];
    svd3(F, U, s, W);
    if (sout) {
        sout[3 * (int64_t)e] = s[0];
        sout[3 * (int64_t)e + 1] = s[1];
        sout[3 * (int64_t)e + 2] = s[2];
    }
    if (Rout) {
        const float one[3] = {1.f, 1.f, 1.f};
        udwt(U, one, W, P);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Rout[9 * (int64_t)e + 3 * i + j] = P[i][j];
    }
    if (Vout) {
        volume_targets(s, d);
        udwt(U, d, W, P);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Vout[9 * (int64_t)e + 3 * i + j] = P[i][j];
    }
}

// geo holds three float4 rows per tet in SoA blocks:
// geo[t] = (g1, ws), geo[n_t + t] = (g2, wv), geo[2 n_t + t] = (g3, 0), with
// g_k the rows of Dm^-1 and ws = V_e gamma_s, wv = V_e gamma_v; the corner
// vectors are g_1, g_2, g_3 and g_0 = -(g1 + g2 + g3).
struct LocalIn {
    float4 r1, r2, r3, x0, x1, x2, x3;
};

// Per-tet corner terms f_c = P g_c with P = U diag(c) W^T: the RHS form
// c_i = w_s + w_v d_i (P = w_s R + w_v V), or the residual form
// c_i = w_s (1 - s_i) + w_v (d_i - s_i) (P = w_s (R - F) + w_v (V - F), the
// elastic part of b - K x without cancellation: F = U diag(s) W^T).
template <bool RESID>
__device__ __forceinline__ void local_corners(const LocalIn& L, float (&out)[4][3]) {
    const float e1[3] = {L.x1.x - L.x0.x, L.x1.y - L.x0.y, L.x1.z - L.x0.z};
    const float e2[3] = {L.x2.x - L.x0.x, L.x2.y - L.x0.y, L.x2.z - L.x0.z};
    const float e3[3] = {L.x3.x - L.x0.x, L.x3.y - L.x0.y, L.x3.z - L.x0.z};
    const float g1[3] = {L.r1.x, L.r1.y, L.r1.z};
    const float g2[3] = {L.r2.x, L.r2.y, L.r2.z};
    const float g3[3] = {L.r3.x, L.r3.y, L.r3.z};
    float F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = e1[i] * g1[j] + e2[i] * g2[j] + e3[i] * g3[j];
    float U[3][3], W[3][3], s[3], d[3], P[3][3];
    svd3(F, U, s, W);
    volume_targets(s, d);
    const float ws = L.r1.w, wv = L.r2.w;
    float c[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) c[i] = RESID ? ws * (1.f - s[i]) + wv * (d[i] - s[i]) : ws + wv * d[i];
    udwt(U, c, W, P);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        out[1][i] = P[i][0] * g1[0] + P[i][1] * g1[1] + P[i][2] * g1[2];
        out[2][i] = P[i][0] * g2[0] + P[i][1] * g2[1] + P[i][2] * g2[2];
        out[3][i] = P[i][0] * g3[0] + P[i][1] * g3[1] + P[i][2] * g3[2];
        out[0][i] = -(out[1][i] + out[2][i] + out[3][i]);
    }
}

// Fused local step and RHS assembly.  Tets are cut into blocks of kLaTets
// consecutive (domain-sorted) tets, one tet per thread; the block's corner
// terms go to shared memory, then every free vertex the block touches sums
// its corners there in increasing (tet, corner) order.  A vertex whose
// corners all lie in one block ("owned") is finished there:
//   RHS form:      b_v = by0_v + sum_c f_c
//   residual form: r_v = (m_v/dt^2)(y_v - x_v) + sum_c f_c  (= b_v - (K x)_v)
// A vertex shared by several blocks gets the block's partial sum in its
// slot (slots ordered by block); k_assemble_shared adds base + the slots in
// slot order (deterministic, no atomics).
constexpr int kLaTets = PDG_LA_TETS;
#ifndef PDG_LA_MINB
#define PDG_LA_MINB 8
#endif

template <bool RESID>
__device__ __forceinline__ float4 assembly_base(const LocalAsmArgs& A, int v) {
    if (RESID) {
        const float m = A.mh2[v];
        const float4 y = A.y[v], xv = A.x[v];
        return make_float4(m * (y.x - xv.x), m * (y.y - xv.y), m * (y.z - xv.z), 0.f);
    }
    return A.by0[v];
}

// One block of the fused kernel: tets [blk kLaTets, (blk + 1) kLaTets) of the mesh in A.
template <bool RESID>
__device__ __forceinline__ void local_assemble_block(const LocalAsmArgs& A, int blk) {
    __shared__ float fx[4 * kLaTets], fy[4 * kLaTets], fz[4 * kLaTets];
    pdl_trigger();
    const int e = blk * kLaTets + threadIdx.x;
    const bool live = e < A.n_t;
    const int ec = live ? e : A.n_t - 1;
    LocalIn L;
    const int4 tv = __ldg(&A.tets[ec]);
    L.r1 = __ldg(&A.geo[ec]);
    L.r2 = __ldg(&A.geo[A.n_t + ec]);
    L.r3 = __ldg(&A.geo[2 * (int64_t)A.n_t + ec]);
    const int j0 = __ldg(&A.vptr[blk]), j1 = __ldg(&A.vptr[blk + 1]);
    pdl_wait();   // x comes from the previous solve
    L.x0 = A.x[tv.x];
    L.x1 = A.x[tv.y];
    L.x2 = A.x[tv.z];
    L.x3 = A.x[tv.w];
    float f[4][3];
    local_corners<RESID>(L, f);
    if (live) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            fx[4 * threadIdx.x + c] = f[c][0];
            fy[4 * threadIdx.x + c] = f[c][1];
            fz[4 * threadIdx.x + c] = f[c][2];
        }
    }
    __syncthreads();
    for (int j = j0 + threadIdx.x; j < j1; j += kLaTets) {
        const int k0 = __ldg(&A.cptr[j]), k1 = __ldg(&A.cptr[j + 1]);
        float ax = 0.f, ay = 0.f, az = 0.f;
        for (int k = k0; k < k1; ++k) {
            const int q = __ldg(&A.corner[k]);
            ax += fx[q];
            ay += fy[q];
            az += fz[q];
        }
        const int slot = __ldg(&A.slot[j]);
        if (slot >= 0) {
            A.part[slot] = make_float4(ax, ay, az, 0.f);
        } else {
            const int v = __ldg(&A.vert[j]);
            const float4 base = assembly_base<RESID>(A, v);
            A.b[v] = make_float4(base.x + ax, base.y + ay, base.z + az, 0.f);
        }
    }
}

template <bool RESID>
__global__ void __launch_bounds__(kLaTets, PDG_LA_MINB) k_local_assemble(LocalAsmArgs A) {
    local_assemble_block<RESID>(A, blockIdx.x);
}

// shared vertices: b_v = base + the blocks' partial sums in block order
template <bool RESID>
__device__ __forceinline__ void assemble_shared_block(const LocalAsmArgs& A, int n_shared, int blk) {
    pdl_trigger();
    const int j = blk * 256 + threadIdx.x;
    const bool live = j < n_shared;
    const int v = live ? __ldg(&A.sh_vert[j]) : 0;
    const int s0 = live ? __ldg(&A.sh_ptr[j]) : 0, s1 = live ? __ldg(&A.sh_ptr[j + 1]) : 0;
    pdl_wait();   // the partial sums come from k_local_assemble
    if (!live) return;
    float4 acc = assembly_base<RESID>(A, v);
    for (int q = s0; q < s1; ++q) {
        const float4 p = A.part[q];
        acc.x += p.x;
        acc.y += p.y;
        acc.z += p.z;
    }
    A.b[v] = make_float4(acc.x, acc.y, acc.z, 0.f);
}

template <bool RESID>
__global__ void __launch_bounds__(256) k_assemble_shared(LocalAsmArgs A, int n_shared) {
    assemble_shared_block<RESID>(A, n_shared, blockIdx.x);
}

// Serving: the same two kernels over every resident request of a batch (RHS
// form); a block finds its request from the per-kernel block offsets, so each
// request's values come from exactly the arithmetic and order above.
__device__ __forceinline__ LocalAsmArgs batch_args(const BatchSlot& S) {
    LocalAsmArgs A{};
    A.n_t = S.n_t;
    A.tets = S.tets;
    A.geo = S.geo;
    A.x = S.x;
    A.by0 = S.by0;
    A.b = S.b;
    A.vptr = S.la_vptr;
    A.vert = S.la_vert;
    A.slot = S.la_slot;
    A.cptr = S.la_cptr;
    A.corner = S.la_corner;
    A.sh_ptr = S.la_sh_ptr;
    A.sh_vert = S.la_sh_vert;
    A.part = S.la_part;
    return A;
}

__global__ void __launch_bounds__(kLaTets, PDG_LA_MINB) k_b_local_assemble(const BatchSlot* __restrict__ slots,
                                                                         const int* __restrict__ off, int n_slots) {
    const int s = batch_find_slot(off, n_slots, blockIdx.x);
    local_assemble_block<false>(batch_args(slots[s]), blockIdx.x - off[s]);
}

__global__ void __launch_bounds__(256) k_b_assemble_shared(const BatchSlot* __restrict__ slots,
                                                         const int* __restrict__ off, int n_slots) {
    const int s = batch_find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    assemble_shared_block<false>(batch_args(S), S.la_shared, blockIdx.x - off[s]);
}

}  // namespace

// Assembly plan of the fused kernel from the tet -> (sorted) vertex table and
// the free-vertex incidence lists (increasing 4 t + c).
void build_local_plan(pd_mesh* m, const std::vector<int32_t>& inc_ptr, const std::vector<int32_t>& inc,
                      cudaStream_t s) {
    const int32_t n_t = m->n_t, n_free = m->n_free;
    const int32_t n_blk = std::max(1, (n_t + kLaTets - 1) / kLaTets);
    // per free vertex: the blocks its corners fall in (ascending, since inc is ascending)
    std::vector<int32_t> sh_of(n_free, -1), sh_ptr(1, 0), sh_vert;
    std::vector<int32_t> cnt_entries(n_blk, 0);
    for (int32_t v = 0; v < n_free; ++v) {
        int32_t nb = 0, last = -1;
        for (int32_t k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
            const int32_t b = (inc[k] / 4) / kLaTets;
            if (b != last) {
                ++nb;
                ++cnt_entries[b];
                last = b;
            }
        }
        if (nb > 1) {
            sh_of[v] = (int32_t)sh_vert.size();
            sh_vert.push_back(v);
            sh_ptr.push_back(sh_ptr.back() + nb);
        }
    }
    std::vector<int32_t> vptr(n_blk + 1, 0);
    for (int32_t b = 0; b < n_blk; ++b) vptr[b + 1] = vptr[b] + cnt_entries[b];
    const int32_t n_ent = vptr[n_blk];
    std::vector<int32_t> vert(n_ent), sidx(n_ent), slot(n_ent), ccount(n_ent, 0), fill(vptr.begin(), vptr.end() - 1);
    // entries in vertex order within each block; corner counts
    for (int32_t v = 0; v < n_free; ++v) {
        int32_t last = -1, rank = 0, j = -1;
        for (int32_t k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
            const int32_t b = (inc[k] / 4) / kLaTets;
            if (b != last) {
                j = fill[b]++;
                vert[j] = v;
                sidx[j] = sh_of[v];
                slot[j] = sh_of[v] < 0 ? -1 : sh_ptr[sh_of[v]] + rank;
                ++rank;
                last = b;
            }
            ++ccount[j];
        }
    }
    std::vector<int32_t> cptr(n_ent + 1, 0);
    for (int32_t j = 0; j < n_ent; ++j) cptr[j + 1] = cptr[j] + ccount[j];
    std::vector<uint16_t> corner(std::max<int32_t>(cptr[n_ent], 1));
    std::fill(ccount.begin(), ccount.end(), 0);
    std::fill(fill.begin(), fill.end(), 0);
    std::copy(vptr.begin(), vptr.end() - 1, fill.begin());
    for (int32_t v = 0; v < n_free; ++v) {
        int32_t last = -1, j = -1;
        for (int32_t k = inc_ptr[v]; k < inc_ptr[v + 1]; ++k) {
            const int32_t b = (inc[k] / 4) / kLaTets;
            if (b != last) {
                j = fill[b]++;
                last = b;
            }
            corner[cptr[j] + ccount[j]++] = (uint16_t)(inc[k] - 4 * b * kLaTets);
        }
    }
    (void)sidx;
    upload(m->d_la_vptr, vptr, s);
    upload(m->d_la_vert, vert, s);
    upload(m->d_la_slot, slot, s);
    upload(m->d_la_cptr, cptr, s);
    upload(m->d_la_corner, corner, s);
    upload(m->d_la_sh_ptr, sh_ptr, s);
    upload(m->d_la_sh_vert, sh_vert, s);
    m->d_la_part.alloc(std::max<size_t>(sh_ptr.back(), 1));
    m->la_blocks = n_blk;
    m->la_entries = n_ent;
    m->la_corners = cptr[n_ent];
    m->la_slots = sh_ptr.back();
    m->la_shared = (int32_t)sh_vert.size();
    PDG_CUDA(cudaStreamSynchronize(s));   // the host vectors are released on return
}

void launch_local_assemble(const pd_mesh* m, const float4* x, const float4* by0, const float4* y, float4* b,
                           bool residual, cudaStream_t s) {
    if (m->n_t <= 0) return;
    LocalAsmArgs A{};
    A.n_t = m->n_t;
    A.tets = m->d_tets.p;
    A.geo = m->d_geo.p;
    A.x = x;
    A.by0 = by0;
    A.y = y;
    A.mh2 = m->d_mh2.p;
    A.b = b;
    A.vptr = m->d_la_vptr.p;
    A.vert = m->d_la_vert.p;
    A.slot = m->d_la_slot.p;
    A.cptr = m->d_la_cptr.p;
    A.corner = m->d_la_corner.p;
    A.sh_ptr = m->d_la_sh_ptr.p;
    A.sh_vert = m->d_la_sh_vert.p;
    A.part = m->d_la_part.p;
    const int nsb = (m->la_shared + 255) / 256;
    if (residual) {
        launch_pdl(k_local_assemble<true>, dim3(m->la_blocks), dim3(kLaTets), 0, s, A);
        if (nsb > 0) launch_pdl(k_assemble_shared<true>, dim3(nsb), dim3(256), 0, s, A, m->la_shared);
    } else {
        launch_pdl(k_local_assemble<false>, dim3(m->la_blocks), dim3(kLaTets), 0, s, A);
        if (nsb > 0) launch_pdl(k_assemble_shared<false>, dim3(nsb), dim3(256), 0, s, A, m->la_shared);
    }
    PDG_CHECK_LAUNCH();
}

void launch_b_local_assemble(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    k_b_local_assemble<<<blocks, kLaTets, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}

void launch_b_assemble_shared(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    k_b_assemble_shared<<<blocks, 256, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}

void launch_project(const float* F, int n, float* R, float* V, float* sig, cudaStream_t s) {
    if (n <= 0) return;
    k_project<<<(n + 255) / 256, 256, 0, s>>>(F, n, R, V, sig);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg

// Batched per-frame kernels of the serving loop: one launch advances every
// resident request ("slot") of the server.  Each slot keeps its own mesh
// arrays and factorisation; a block finds its slot from per-kernel block
// offsets, so each slot's values are computed with exactly the arithmetic
// and summation order of the single-mesh kernels (results do not depend on
// which other requests share the launch).
#include "pd_internal.h"
#include "proj3.cuh"

namespace pdg {

namespace {

using namespace proj;

__device__ __forceinline__ int find_slot(const int* __restrict__ off, int n, int b) {
    // last s with off[s] <= b  (off[0] = 0, off increasing)
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float4 f4(float x, float y, float z) { return make_float4(x, y, z, 0.f); }

// pinned targets for the coming frame: rest + amp sin(w t) e_axis, t = (frame + 1) h
__global__ void k_b_drive(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    const int k = (blockIdx.x - off[s]) * blockDim.x + threadIdx.x;
    if (k >= S.n_pin) return;
    const float t = (float)(S.frame[0] + 1) * S.h;
    const float d = S.drive_amp * sinf(S.drive_w * t);
    float4 p = S.pin_rest[k];
    if (S.drive_axis == 0) p.x += d;
    else if (S.drive_axis == 1) p.y += d;
    else p.z += d;
    S.pin_tgt[k] = p;
}

__global__ void k_b_inertia(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    const int i = (blockIdx.x - off[s]) * blockDim.x + threadIdx.x;
    if (i >= S.n_v) return;
    const float4 xp = S.x[i];
    S.xprev[i] = xp;
    if (i < S.n_free) {
        const float4 vv = S.v[i];
        const float h = S.h, h2 = h * h;
        const float4 y = f4(xp.x + h * vv.x + h2 * S.gx, xp.y + h * vv.y + h2 * S.gy, xp.z + h * vv.z + h2 * S.gz);
        S.x[i] = y;
        const float m = S.mh2[i];
        float4 acc = f4(m * y.x, m * y.y, m * y.z);
        for (int k = S.kfp_ptr[i]; k < S.kfp_ptr[i + 1]; ++k) {
            const float kv = S.kfp_val[k];
            const float4 p = S.pin_tgt[S.kfp_col[k]];
            acc.x -= kv * p.x;
            acc.y -= kv * p.y;
            acc.z -= kv * p.z;
        }
        S.by0[i] = acc;
    } else {
        S.x[i] = S.pin_tgt[i - S.n_free];
    }
}

__global__ void __launch_bounds__(128) k_b_local(const BatchSlot* __restrict__ slots, const int* __restrict__ off,
                                                 int n_slots) {
    const int s = find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    const int e = (blockIdx.x - off[s]) * blockDim.x + threadIdx.x;
    if (e >= S.n_t) return;
    const int n_t = S.n_t;
    const int4 tv = __ldg(&S.tets[e]);
    const float4 r1 = __ldg(&S.geo[e]);
    const float4 r2 = __ldg(&S.geo[n_t + e]);
    const float4 r3 = __ldg(&S.geo[2 * (int64_t)n_t + e]);
    const float4 x0 = S.x[tv.x], x1 = S.x[tv.y], x2 = S.x[tv.z], x3 = S.x[tv.w];
    const float e1[3] = {x1.x - x0.x, x1.y - x0.y, x1.z - x0.z};
    const float e2[3] = {x2.x - x0.x, x2.y - x0.y, x2.z - x0.z};
    const float e3[3] = {x3.x - x0.x, x3.y - x0.y, x3.z - x0.z};
    const float g1[3] = {r1.x, r1.y, r1.z};
    const float g2[3] = {r2.x, r2.y, r2.z};
    const float g3[3] = {r3.x, r3.y, r3.z};
    float F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F[i][j] = e1[i] * g1[j] + e2[i] * g2[j] + e3[i] * g3[j];
    float U[3][3], W[3][3], sv[3], d[3], P[3][3];
    svd3(F, U, sv, W);
    volume_targets(sv, d);
    const float ws = r1.w, wv = r2.w;
    const float c[3] = {ws + wv * d[0], ws + wv * d[1], ws + wv * d[2]};
    udwt(U, c, W, P);
    float f1[3], f2[3], f3[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        f1[i] = P[i][0] * g1[0] + P[i][1] * g1[1] + P[i][2] * g1[2];
        f2[i] = P[i][0] * g2[0] + P[i][1] * g2[1] + P[i][2] * g2[2];
        f3[i] = P[i][0] * g3[0] + P[i][1] * g3[1] + P[i][2] * g3[2];
    }
    float4* out = S.force + 4 * (int64_t)e;
    out[0] = f4(-(f1[0] + f2[0] + f3[0]), -(f1[1] + f2[1] + f3[1]), -(f1[2] + f2[2] + f3[2]));
    out[1] = f4(f1[0], f1[1], f1[2]);
    out[2] = f4(f2[0], f2[1], f2[2]);
    out[3] = f4(f3[0], f3[1], f3[2]);
}

__global__ void __launch_bounds__(256) k_b_assemble(const BatchSlot* __restrict__ slots, const int* __restrict__ off,
                                                    int n_slots) {
    const int s = find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    const int i = (blockIdx.x - off[s]) * blockDim.x + threadIdx.x;
    if (i >= S.n_free) return;
    float4 acc = S.by0[i];
    const int k0 = S.inc_ptr[i], k1 = S.inc_ptr[i + 1];
    int k = k0;
    for (; k + 4 <= k1; k += 4) {
        const int a0 = S.inc[k], a1 = S.inc[k + 1], a2 = S.inc[k + 2], a3 = S.inc[k + 3];
        const float4 q0 = S.force[a0], q1 = S.force[a1], q2 = S.force[a2], q3 = S.force[a3];
        acc.x += q0.x; acc.y += q0.y; acc.z += q0.z;
        acc.x += q1.x; acc.y += q1.y; acc.z += q1.z;
        acc.x += q2.x; acc.y += q2.y; acc.z += q2.z;
        acc.x += q3.x; acc.y += q3.y; acc.z += q3.z;
    }
    for (; k < k1; ++k) {
        const float4 q0 = S.force[S.inc[k]];
        acc.x += q0.x; acc.y += q0.y; acc.z += q0.z;
    }
    S.b[i] = acc;
}

__global__ void k_b_gather(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    const int j = (blockIdx.x - off[s]) * blockDim.x + threadIdx.x;
    if (j >= S.n_B) return;
    float4 acc = S.b[S.n_int + j];
    for (int k = S.gat_ptr[j]; k < S.gat_ptr[j + 1]; ++k) {
        const float4 c = S.tc[S.gat[k]];
        acc.x += c.x; acc.y += c.y; acc.z += c.z;
    }
    S.cB[j] = acc;
}

__global__ void k_b_reduce(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    const int j = (blockIdx.x - off[s]) * blockDim.x + threadIdx.x;
    if (j >= S.n_B) return;
    float4 acc = S.part[j];
    for (int c = 1; c < S.nch; ++c) {
        const float4 p = S.part[(int64_t)c * S.n_B + j];
        acc.x += p.x; acc.y += p.y; acc.z += p.z;
    }
    S.x[S.n_int + j] = make_float4(acc.x, acc.y, acc.z, 0.f);
}

__global__ void k_b_velocity(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    const int i = (blockIdx.x - off[s]) * blockDim.x + threadIdx.x;
    if (i == 0 && blockIdx.x == off[s]) {
        // the frame counter advances once per frame (read by the next frame's drive kernel)
        S.frame[0] += 1;
    }
    if (i >= S.n_v) return;
    const float4 a = S.x[i], b = S.xprev[i];
    const float ih = 1.0f / S.h;
    const float4 vv = f4((a.x - b.x) * ih, (a.y - b.y) * ih, (a.z - b.z) * ih);
    S.v[i] = vv;
    if (!(isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(vv.x) && isfinite(vv.y) && isfinite(vv.z)))
        atomicOr(S.err, ERR_NONFINITE);
}

inline int nblk(int n, int b) { return (n + b - 1) / b; }

}  // namespace

// The launches of one batched frame phase; `off` = device block offsets for that phase.
void launch_b_drive(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    k_b_drive<<<blocks, 256, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}
void launch_b_inertia(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    k_b_inertia<<<blocks, 256, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}
void launch_b_local(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    k_b_local<<<blocks, 128, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}
void launch_b_assemble(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    k_b_assemble<<<blocks, 256, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}
void launch_b_gather(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    k_b_gather<<<blocks, 256, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}
void launch_b_reduce(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    k_b_reduce<<<blocks, 256, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}
void launch_b_velocity(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    k_b_velocity<<<blocks, 256, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg

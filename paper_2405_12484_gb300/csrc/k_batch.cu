// Batched per-frame kernels of the serving loop: one launch advances every
// resident request ("slot") of the server.  Each slot keeps its own mesh
// arrays and factorisation; a block finds its slot from per-kernel block
// offsets, so each slot's values are computed with exactly the arithmetic
// and summation order of the single-mesh kernels (results do not depend on
// which other requests share the launch).  The local step and assembly of
// a batch are the fused kernels of the single-mesh frame (k_local.cu).
#include "pd_internal.h"

namespace pdg {

namespace {

__device__ __forceinline__ float4 f4(float x, float y, float z) { return make_float4(x, y, z, 0.f); }

// pinned targets for the coming frame: rest + amp sin(w t) e_axis, t = (frame + 1) h
__global__ void k_b_drive(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = batch_find_slot(off, n_slots, blockIdx.x);
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
    const int s = batch_find_slot(off, n_slots, blockIdx.x);
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

__global__ void k_b_gather(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = batch_find_slot(off, n_slots, blockIdx.x);
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

// two-level requests: c_T = c_B[T0:] + the gathered second-level terms (as k_gather)
__global__ void k_b_gather2(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = batch_find_slot(off, n_slots, blockIdx.x);
    const BatchSlot& S = slots[s];
    const int j = (blockIdx.x - off[s]) * blockDim.x + threadIdx.x;
    if (j >= S.n_top) return;
    float4 acc = S.cB[S.n_B - S.n_top + j];
    for (int k = S.gat2_ptr[j]; k < S.gat2_ptr[j + 1]; ++k) {
        const float4 c = S.tc2[S.gat2[k]];
        acc.x += c.x; acc.y += c.y; acc.z += c.z;
    }
    S.cT[j] = acc;
}

__global__ void k_b_reduce(const BatchSlot* __restrict__ slots, const int* __restrict__ off, int n_slots) {
    const int s = batch_find_slot(off, n_slots, blockIdx.x);
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
    const int s = batch_find_slot(off, n_slots, blockIdx.x);
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
void launch_b_gather(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    k_b_gather<<<blocks, 256, 0, s>>>(slots, off, n_slots);
    PDG_CHECK_LAUNCH();
}
void launch_b_gather2(const BatchSlot* slots, const int* off, int n_slots, int blocks, cudaStream_t s) {
    if (blocks <= 0) return;
    k_b_gather2<<<blocks, 256, 0, s>>>(slots, off, n_slots);
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

// Per-vertex kernels of the PD frame: inertial target, deterministic RHS
// assembly (segmented gather, no float atomics), velocity update, and the
// permutations between the caller's vertex order and the library's.
//
// Paper: Sec. 7 (implicit Euler: a = x - x* - dt v* - dt^2 M^-1 f, so the
// inertial target is y = x* + dt v* + dt^2 g), Sec. 7.1 (b = (M/dt^2) y +
// sum_e V_e gs B^T (D^T:R) + sum_e V_e gv B^T (D^T:V)).
#include "pd_internal.h"

namespace pdg {

namespace {

__device__ __forceinline__ float4 f4(float x, float y, float z) { return make_float4(x, y, z, 0.f); }

// x* <- x; free vertices: y = x* + h v + h^2 g, x^0 = y and
// by0 = (m/h^2) y - sum_p K_fp x_p; pinned vertices: x = target.
__global__ void k_inertia(int n_v, int n_free, float h, float gx, float gy, float gz, float4* __restrict__ x,
                          float4* __restrict__ xprev, const float4* __restrict__ v, const float4* __restrict__ tgt,
                          const float* __restrict__ mh2, const int* __restrict__ kfp_ptr,
                          const int* __restrict__ kfp_col, const float* __restrict__ kfp_val,
                          float4* __restrict__ by0, float4* __restrict__ yout) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v) return;
    float4 xp = x[i];
    xprev[i] = xp;
    if (i < n_free) {
        float4 vv = v[i];
        float h2 = h * h;
        float4 y = f4(xp.x + h * vv.x + h2 * gx, xp.y + h * vv.y + h2 * gy, xp.z + h * vv.z + h2 * gz);
        x[i] = y;
        if (yout) yout[i] = y;
        float m = mh2[i];
        float4 acc = f4(m * y.x, m * y.y, m * y.z);
        for (int k = kfp_ptr[i]; k < kfp_ptr[i + 1]; ++k) {
            float kv = kfp_val[k];
            float4 p = tgt[kfp_col[k]];
            acc.x -= kv * p.x;
            acc.y -= kv * p.y;
            acc.z -= kv * p.z;
        }
        by0[i] = acc;
    } else {
        x[i] = tgt[i - n_free];
    }
}

// by0 = (m/h^2) y - K_fp x_p for a given y (diagnostic path); pinned x_p from x.
__global__ void k_by0(int n_free, const float4* __restrict__ y, const float4* __restrict__ xpin,
                      const float* __restrict__ mh2, const int* __restrict__ kfp_ptr, const int* __restrict__ kfp_col,
                      const float* __restrict__ kfp_val, float4* __restrict__ by0) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_free) return;
    float4 yy = y[i];
    float m = mh2[i];
    float4 acc = f4(m * yy.x, m * yy.y, m * yy.z);
    for (int k = kfp_ptr[i]; k < kfp_ptr[i + 1]; ++k) {
        float kv = kfp_val[k];
        float4 p = xpin[kfp_col[k]];
        acc.x -= kv * p.x;
        acc.y -= kv * p.y;
        acc.z -= kv * p.z;
    }
    by0[i] = acc;
}

__global__ void k_velocity(int n_v, float inv_h, const float4* __restrict__ x, const float4* __restrict__ xprev,
                           float4* __restrict__ v, int* __restrict__ err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v) return;
    float4 a = x[i], b = xprev[i];
    float4 vv = f4((a.x - b.x) * inv_h, (a.y - b.y) * inv_h, (a.z - b.z) * inv_h);
    v[i] = vv;
    if (!(isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(vv.x) && isfinite(vv.y) && isfinite(vv.z)))
        atomicOr(err, ERR_NONFINITE);
}

// user pinned targets (n_pin x 3, increasing vertex id) -> internal pinned slots
__global__ void k_pin_copy(int n_pin, const float* __restrict__ src, float4* __restrict__ tgt) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pin) return;
    tgt[k] = f4(src[3 * k], src[3 * k + 1], src[3 * k + 2]);
}

__global__ void k_pin_hold(int n_pin, int n_free, const float4* __restrict__ x, float4* __restrict__ tgt) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pin) return;
    tgt[k] = x[n_free + k];
}

// dst[old] = src[new] (n_v x 3); free_only: pinned rows are written as 0
__global__ void k_scatter_out(int n_v, int n_free, const int* __restrict__ old_of_new, const float4* __restrict__ src,
                              float* __restrict__ dst, int free_only) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v) return;
    float4 a = (free_only && i >= n_free) ? f4(0.f, 0.f, 0.f) : src[i];
    int o = old_of_new[i];
    dst[3 * (int64_t)o] = a.x;
    dst[3 * (int64_t)o + 1] = a.y;
    dst[3 * (int64_t)o + 2] = a.z;
}

// dst[new] = src[old]
__global__ void k_gather_in(int n_v, const int* __restrict__ old_of_new, const float* __restrict__ src,
                            float4* __restrict__ dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v) return;
    int o = old_of_new[i];
    dst[i] = f4(src[3 * (int64_t)o], src[3 * (int64_t)o + 1], src[3 * (int64_t)o + 2]);
}

// geo[t].w = V_e gamma_s, geo[n_t + t].w = V_e gamma_v (inputs already in sorted tet order)
__global__ void k_weights(int n_t, const float* __restrict__ vol, const float* __restrict__ gs,
                          const float* __restrict__ gv, float4* __restrict__ geo) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_t) return;
    geo[t].w = vol[t] * gs[t];
    geo[n_t + t].w = vol[t] * gv[t];
}

inline int nblk(int n, int b) { return (n + b - 1) / b; }

}  // namespace

void launch_inertia(const pd_mesh* m, float h, float gx, float gy, float gz, cudaStream_t s) {
    k_inertia<<<nblk(m->n_v, 256), 256, 0, s>>>(m->n_v, m->n_free, h, gx, gy, gz, m->d_x.p, m->d_xprev.p, m->d_v.p,
                                                m->d_pin_tgt.p, m->d_mh2.p, m->d_kfp_ptr.p, m->d_kfp_col.p,
                                                m->d_kfp_val.p, m->d_by0.p, m->correction ? m->d_y.p : nullptr);
    PDG_CHECK_LAUNCH();
}

void launch_by0_from_y(const pd_mesh* m, const float4* y, float4* by0, cudaStream_t s) {
    if (m->n_free <= 0) return;
    // pinned positions come from the pin-target buffer (filled by the caller)
    k_by0<<<nblk(m->n_free, 256), 256, 0, s>>>(m->n_free, y, m->d_pin_tgt.p, m->d_mh2.p, m->d_kfp_ptr.p,
                                               m->d_kfp_col.p, m->d_kfp_val.p, by0);
    PDG_CHECK_LAUNCH();
}

void launch_velocity(const pd_mesh* m, float inv_h, cudaStream_t s) {
    k_velocity<<<nblk(m->n_v, 256), 256, 0, s>>>(m->n_v, inv_h, m->d_x.p, m->d_xprev.p, m->d_v.p, m->d_err.p);
    PDG_CHECK_LAUNCH();
}

void launch_pin_copy(const pd_mesh* m, const float* user_targets, cudaStream_t s) {
    if (m->n_pin <= 0) return;
    k_pin_copy<<<nblk(m->n_pin, 256), 256, 0, s>>>(m->n_pin, user_targets, m->d_pin_tgt.p);
    PDG_CHECK_LAUNCH();
}

void launch_pin_hold(const pd_mesh* m, cudaStream_t s) {
    if (m->n_pin <= 0) return;
    k_pin_hold<<<nblk(m->n_pin, 256), 256, 0, s>>>(m->n_pin, m->n_free, m->d_x.p, m->d_pin_tgt.p);
    PDG_CHECK_LAUNCH();
}

void launch_scatter_out(const pd_mesh* m, const float4* src, float* dst, int free_only, cudaStream_t s) {
    k_scatter_out<<<nblk(m->n_v, 256), 256, 0, s>>>(m->n_v, m->n_free, m->d_old_of_new.p, src, dst, free_only);
    PDG_CHECK_LAUNCH();
}

void launch_gather_in(const pd_mesh* m, const float* src, float4* dst, cudaStream_t s) {
    k_gather_in<<<nblk(m->n_v, 256), 256, 0, s>>>(m->n_v, m->d_old_of_new.p, src, dst);
    PDG_CHECK_LAUNCH();
}

void launch_weights_raw(int n_t, const float* vol, const float* gs, const float* gv, float4* geo, cudaStream_t s) {
    k_weights<<<nblk(n_t, 256), 256, 0, s>>>(n_t, vol, gs, gv, geo);
    PDG_CHECK_LAUNCH();
}

}  // namespace pdg

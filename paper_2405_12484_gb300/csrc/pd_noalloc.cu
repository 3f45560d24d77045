// pd_solve_noalloc: the subspace global solve of pd_solve with every
// temporary taken from one fixed, statically allocated device array instead
// of cudaMalloc.
//
// Who needs it: callers that may not allocate device memory while they run
// (for example a host that sub-allocates a fixed memory pool to every
// library and forbids cudaMalloc/cudaFree after start-up, or code running
// inside a region where allocation would synchronise the device).  After
// pd_prefactor has run, this entry point needs no allocation at all.
//
// The scratch array is a file-scope __device__ array of kNoallocBytes
// (16 MiB).  Every GPU on which this library is loaded holds it until the
// process exits.  Host code must not use the array's name as a device
// address; its device address is obtained once per device with
// cudaGetSymbolAddress.  That lookup loads this file's device module (the
// CUDA runtime loads modules lazily), which is when the 16 MiB is actually
// taken from the device; pd_prefactor therefore makes it, on the mesh's
// device, while allocation is still allowed, and pd_solve_noalloc itself
// only reads the cached address.  A call on a device where no pd_prefactor
// has run yet makes the lookup itself (and so may take the 16 MiB then);
// such a first call must come before any stream capture.
#include <mutex>

#include "pd_internal.h"

namespace pdg {

void launch_dd_solve_scratch(pd_mesh* m, const float4* b, float4* xout, float4* tc, float4* cB, float4* part,
                             float4* tc2, float4* cT, float4* xg2, float4* xgB, float4* pm, float4* jx1, float4* jx2,
                             cudaStream_t s);

namespace {

constexpr size_t kNoallocBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up and
// cached on first use).  Returns nullptr after recording the error.
unsigned char* scratch_base(pd_status* code) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("pd_solve_noalloc: cudaGetDevice failed: ") + cudaGetErrorString(e));
        *code = PD_ERR_CUDA;
        return nullptr;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("pd_solve_noalloc: device ordinal out of range");
        *code = PD_ERR_UNSUPPORTED;
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            (void)cudaGetLastError();
            set_error(std::string("pd_solve_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            *code = PD_ERR_CUDA;
            return nullptr;
        }
        g_scratch_addr[dev] = p;
    }
    return static_cast<unsigned char*>(g_scratch_addr[dev]);
}

}  // namespace

// Called by pd_prefactor on the mesh's device: resolves (and so loads) the
// scratch array there, so that later pd_solve_noalloc calls take no device
// memory at all.
pd_status noalloc_prepare_device() {
    pd_status code = PD_OK;
    return scratch_base(&code) ? PD_OK : code;
}

}  // namespace pdg

using namespace pdg;

extern "C" pd_status pd_solve_noalloc(pd_mesh* m, const float* r, float* x) {
    if (!m || !r || !x) {
        set_error("pd_solve_noalloc: null argument");
        return PD_ERR_INVALID_ARG;
    }
    if (!m->prefactored) {
        set_error("pd_solve_noalloc: pd_prefactor has not run");
        return PD_ERR_NOT_PREFACTORED;
    }
    // layout of the shared scratch: inputs/outputs in library order, the
    // per-domain condensed rows, the interface right-hand side, the coarse
    // partial sums, and the refinement residual and correction
    const size_t nv = (size_t)m->n_v, nf = (size_t)(m->n_free > 0 ? m->n_free : 1);
    const size_t ntc = (size_t)(m->n_tc > 0 ? m->n_tc : 1), nb = (size_t)(m->n_B > 0 ? m->n_B : 1);
    const size_t ncs = (size_t)(m->cs_n > 0 ? m->cs_n : 1);
    const size_t npart = ncs * (size_t)(m->coarse_nchunks > 0 ? m->coarse_nchunks : 1);
    const size_t ntc2 = (size_t)(m->n_tc2 > 0 ? m->n_tc2 : 1), ntop = (size_t)(m->n_top > 0 ? m->n_top : 1);
    const size_t off_r = 0;
    const size_t off_x = off_r + align256(nv * sizeof(float4));
    const size_t off_tc = off_x + align256(nv * sizeof(float4));
    const size_t off_cb = off_tc + align256(ntc * sizeof(float4));
    const size_t off_part = off_cb + align256(nb * sizeof(float4));
    const size_t off_rr = off_part + align256(npart * sizeof(float4));
    const size_t off_dx = off_rr + align256(nf * sizeof(float4));
    const size_t off_tc2 = off_dx + align256(nv * sizeof(float4));
    const size_t off_ct = off_tc2 + align256(ntc2 * sizeof(float4));
    const size_t nxg2 = (size_t)(m->n_xg2 > 0 ? m->n_xg2 : 1), nxgb = (size_t)(m->n_xgB > 0 ? m->n_xgB : 1);
    const size_t off_xg2 = off_ct + align256(ntop * sizeof(float4));
    const size_t off_xgb = off_xg2 + align256(nxg2 * sizeof(float4));
    const size_t npm = (size_t)(m->n_pm > 0 ? m->n_pm : 1);
    const size_t njx = m->jacobi_omega.empty() ? 1 : nf;
    const size_t off_pm = off_xgb + align256(nxgb * sizeof(float4));
    const size_t off_jx1 = off_pm + align256(npm * sizeof(float4));
    const size_t off_jx2 = off_jx1 + align256(njx * sizeof(float4));
    const size_t total = off_jx2 + align256(njx * sizeof(float4));
    if (total > kNoallocBytes) {
        set_error("pd_solve_noalloc: this mesh needs " + std::to_string(total) +
                  " bytes of scratch, more than the fixed 16 MiB (16777216 bytes); use pd_solve");
        return PD_ERR_UNSUPPORTED;
    }
    try {
        pd_status code = PD_OK;
        unsigned char* base = scratch_base(&code);
        if (!base) return code;
        float4* ri = reinterpret_cast<float4*>(base + off_r);
        float4* xi = reinterpret_cast<float4*>(base + off_x);
        float4* tc = reinterpret_cast<float4*>(base + off_tc);
        float4* cB = reinterpret_cast<float4*>(base + off_cb);
        float4* part = reinterpret_cast<float4*>(base + off_part);
        float4* rr = reinterpret_cast<float4*>(base + off_rr);
        float4* dx = reinterpret_cast<float4*>(base + off_dx);
        float4* tc2 = reinterpret_cast<float4*>(base + off_tc2);
        float4* cT = reinterpret_cast<float4*>(base + off_ct);
        float4* xg2 = reinterpret_cast<float4*>(base + off_xg2);
        float4* xgb = reinterpret_cast<float4*>(base + off_xgb);
        float4* pm = reinterpret_cast<float4*>(base + off_pm);
        float4* jx1 = reinterpret_cast<float4*>(base + off_jx1);
        float4* jx2 = reinterpret_cast<float4*>(base + off_jx2);
        cudaStream_t s = m->stream;
        // the solution buffer keeps the previous call's contents: clear it
        PDG_CUDA(cudaMemsetAsync(xi, 0, nv * sizeof(float4), s));
        launch_gather_in(m, r, ri, s);
        launch_dd_solve_scratch(m, ri, xi, tc, cB, part, tc2, cT, xg2, xgb, pm, jx1, jx2, s);
        for (int k = 0; k < m->refine; ++k) {
            launch_residual(m, ri, xi, rr, s);
            launch_dd_solve_scratch(m, rr, dx, tc, cB, part, tc2, cT, xg2, xgb, pm, jx1, jx2, s);
            launch_axpy_free(m, dx, xi, s);
        }
        launch_scatter_out(m, xi, x, 1, s);
        PDG_CUDA(cudaStreamSynchronize(s));
        return PD_OK;
    } catch (const Fail& f) {
        return f.code;
    } catch (...) {
        set_error("pd_solve_noalloc: unexpected host exception");
        return PD_ERR_CUDA;
    }
}

// api_sph.cu -- C ABI of the neighbour search / SPH density on the octree
// (paper Sect. 3: the tree structure also serves neighbour search and
// smoothed particle hydrodynamics).  The groups and the traversal are the
// gravity walk's; the opening rule and the kernel are the neighbour
// search's (k_sph_walk in k_walk.cu).
#include <string>

#include "common.cuh"

using namespace bonsai;

namespace bonsai {

// Smoothing lengths from caller order to sorted order.
__global__ void k_gather_h(const float *__restrict__ h, const uint32_t *__restrict__ id, int n, float *hs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) hs[i] = h[id[i]];
}

// Density and neighbour count from sorted to caller order.
__global__ void k_scatter_sph(const float *__restrict__ rho_s, const int32_t *__restrict__ cnt_s,
                              const uint32_t *__restrict__ id, int n, float *rho, int32_t *cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t j = id[i];
    if (rho) rho[j] = rho_s[i];
    if (cnt) cnt[j] = cnt_s[i];
}

__global__ void k_sph_reset(DevState *st) {
    if (threadIdx.x == 0) st->walk_next = 0u;
}

}  // namespace bonsai

static int sfail(bonsai_ctx *ctx, int code, const std::string &what, cudaError_t e = cudaSuccess) {
    cudaGetLastError();
    std::string s = what;
    if (e != cudaSuccess) { s += ": "; s += cudaGetErrorString(e); }
    if (ctx) ctx->c.err = s;
    return code;
}

extern "C" {

int bonsai_sph_density(bonsai_ctx *ctx, const float *h, float *rho, int32_t *nngb, int on_device) {
    if (!ctx || !h) return BONSAI_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (!c.built || !c.tree_fresh)
        return sfail(ctx, BONSAI_ERR_NOT_READY, "bonsai_sph_density: needs a tree built from the current positions "
                                                "(bonsai_build or bonsai_step)");
    const int n = (int)c.n;
    // scratch in the learned path's feature array (12 floats per body):
    // sorted h, sorted density, sorted counts, caller-order copies for host output
    float *hs = c.feat, *rho_s = c.feat + c.n, *hin = c.feat + 3 * c.n;
    int32_t *cnt_s = reinterpret_cast<int32_t *>(c.feat + 2 * c.n);
    float *rho_o = c.feat + 4 * c.n;
    int32_t *cnt_o = reinterpret_cast<int32_t *>(c.feat + 5 * c.n);
    cudaError_t e = cudaSuccess;
    const float *hd = h;
    if (!on_device) {
        e = cudaMemcpyAsync(hin, h, 4 * (size_t)n, cudaMemcpyHostToDevice, c.stream);
        hd = hin;
    }
    const int grid = (n + 255) / 256;
    if (e == cudaSuccess) { k_gather_h<<<grid, 256, 0, c.stream>>>(hd, c.id, n, hs); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = launch_cell_cubes(c);
    if (e == cudaSuccess) { k_sph_reset<<<1, 32, 0, c.stream>>>(c.st); e = cudaGetLastError(); }
    if (e == cudaSuccess) e = launch_sph_walk(c, hs, c.cext, rho_s, cnt_s);
    if (e == cudaSuccess && (rho || nngb)) {
        if (on_device) {
            k_scatter_sph<<<grid, 256, 0, c.stream>>>(rho_s, cnt_s, c.id, n, rho, nngb);
            e = cudaGetLastError();
        } else {
            k_scatter_sph<<<grid, 256, 0, c.stream>>>(rho_s, cnt_s, c.id, n, rho_o, cnt_o);
            e = cudaGetLastError();
            if (e == cudaSuccess && rho)
                e = cudaMemcpyAsync(rho, rho_o, 4 * (size_t)n, cudaMemcpyDeviceToHost, c.stream);
            if (e == cudaSuccess && nngb)
                e = cudaMemcpyAsync(nngb, cnt_o, 4 * (size_t)n, cudaMemcpyDeviceToHost, c.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        }
    }
    if (e != cudaSuccess) return sfail(ctx, BONSAI_ERR_CUDA, "bonsai_sph_density", e);
    return BONSAI_OK;
}

}  // extern "C"

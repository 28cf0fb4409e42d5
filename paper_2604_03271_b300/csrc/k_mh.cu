// k_mh.cu -- tile dispatch and launch of the fused FP32 Metropolis kernels
// (k_mh_impl.cuh, instantiated per family in k_mh_{gauss,lor,pv}.cu; the
// coupled-grid kernel of k_mh_full.cuh in k_mh_full_{gauss,lor,pv}.cu).
#include "kernels.h"

namespace smc {

typedef void (*mh_fn)(JobDev *, const int *, int);
mh_fn mh_pick_gauss(int J, int G, int R);
mh_fn mh_pick_lor(int J, int G, int R);
mh_fn mh_pick_pv(int J, int G, int R);
mh_fn mhf_pick_gauss(int J, int G);
mh_fn mhf_pick_lor(int J, int G);
mh_fn mhf_pick_pv(int J, int G);
mh_fn mhp_pick(int J, int G);

static int block_threads(int G) { return G <= 4 ? 128 : 32 * G; }

// CTAs per chain: the phase kernel spreads chains of more than 16 warps over
// a thread-block cluster of 8-warp CTAs
static int cluster_of(int family, int G)
{
    return ((family & (MH_COUPLED - 1)) == FAM_XRD && G > 16) ? G / 8 : 1;
}

// family: FAM_* of the peaks, plus MH_COUPLED for the coupled-grid kernel;
// R: register budget of the fused kernel's tile (0: its default)
static mh_fn pick(int family, int J, int G, int R)
{
    const int fam = family & (MH_COUPLED - 1);
    if (R != 0 && (family & MH_COUPLED)) return nullptr;
    if (fam == FAM_XRD) return (family & MH_COUPLED) ? mhp_pick(J, G) : nullptr;
    if (family & MH_COUPLED) {
        if (fam == FAM_GAUSS) return mhf_pick_gauss(J, G);
        if (fam == FAM_LORENTZ) return mhf_pick_lor(J, G);
        return mhf_pick_pv(J, G);
    }
    if (fam == FAM_GAUSS) return mh_pick_gauss(J, G, R);
    if (fam == FAM_LORENTZ) return mh_pick_lor(J, G, R);
    return mh_pick_pv(J, G, R);
}

bool mh_tile_supported(int family, int J, int G, int R) { return pick(family, J, G, R) != nullptr; }

// Dynamic shared memory of the phase kernel's profile cache: the two parts of
// kcap profiles at every point of the block (threads x J points), if at most 96 KB
static size_t mh_smem(int family, int J, int G, int kcap)
{
    if ((family & (MH_COUPLED - 1)) != FAM_XRD || kcap < 1) return 0;
    const int threads = cluster_of(family, G) > 1 ? 256 : block_threads(G);
    const size_t b = 2 * (size_t)kcap * threads * J * sizeof(float);
    return b <= 96 * 1024 ? b : 0;
}

static cudaLaunchConfig_t cluster_config(int C, int grid, size_t smem, cudaStream_t s, cudaLaunchAttribute *attr)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int mh_resident_grid(int family, int J, int G, int R, int kcap)
{
    mh_fn f = pick(family, J, G, R);
    if (!f) return 0;
    const int C = cluster_of(family, G);
    const size_t smem = mh_smem(family, J, G, kcap);
    // static plus dynamic shared memory may pass 48 KB: opt in for every size
    if (smem > 0) cudaFuncSetAttribute((const void *)f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (C > 1) {
        // clusters of C CTAs resident at once (every CTA of a cluster runs the
        // same chain, so the grid holds whole clusters)
        if (C > 8) cudaFuncSetAttribute((const void *)f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config(C, C * 148, smem, nullptr, attr);
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, (const void *)f, &cfg) != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            return 0;
        }
        return ncl * C;
    }
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void *)f, block_threads(G), smem);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_mh(JobDev *jobs, const int *slots, int nslots, int family, int J, int G, int R,
                      int grid, cudaStream_t s, int kcap)
{
    mh_fn f = pick(family, J, G, R);
    if (!f) return cudaErrorInvalidValue;
    if (nslots <= 0) return cudaSuccess;
    if (grid <= 0) grid = mh_resident_grid(family, J, G, R, kcap);
    const int C = cluster_of(family, G);
    const size_t smem = mh_smem(family, J, G, kcap);
    if (C > 1) {
        if (grid < C || grid % C != 0) return cudaErrorInvalidConfiguration;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config(C, grid, smem, s, attr);
        return cudaLaunchKernelEx(&cfg, f, jobs, slots, nslots);
    }
    f<<<grid, block_threads(G), smem, s>>>(jobs, slots, nslots);
    return cudaGetLastError();
}

}  // namespace smc

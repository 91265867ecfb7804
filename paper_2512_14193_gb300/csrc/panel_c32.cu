// Register-row panel kernel (C32 instantiations) and the cluster-size query; the lane-per-column
// panel kernel is in panel_lc.cu.
#include "lu_internal.cuh"

namespace lu_detail {
namespace {

template <class V, int NBP, int RPT>
cudaError_t launch_panel_t(cudaStream_t s, V A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info,
                           int J, int jb, SwapMap* mi, SwapMap* mb, int* perm) {
    auto kern = panel_kernel<V, NBP, RPT>;
    if (ps.CL > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ps.CL, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ps.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, A, j0, m, ib, ps.R, ipiv, info, J, jb, mi, mb, perm);
}


template <class V>
int query_cluster_max() {
    // largest cluster size (16 or 8) the device will co-schedule for the panel kernel
    auto kern = panel_kernel<V, std::is_same<V, C32>::value ? 32 : 16, 1>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(PANEL_THREADS, 1, 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    return ncl >= 1 ? 16 : 8;
}


}  // namespace

cudaError_t launch_panel(cudaStream_t s, C32 A, const PanelShape& ps, int j0, int m, int ib, int* ipiv, int* info,
                         int J, int jb, SwapMap* mi, SwapMap* mb, int* perm) {
    if (ps.RPT == 1) return launch_panel_t<C32, 32, 1>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
    if (ps.RPT == 2) return launch_panel_t<C32, 16, 2>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
    return launch_panel_t<C32, 8, 4>(s, A, ps, j0, m, ib, ipiv, info, J, jb, mi, mb, perm);
}

int query_cluster_max_c32() { return query_cluster_max<C32>(); }

}  // namespace lu_detail

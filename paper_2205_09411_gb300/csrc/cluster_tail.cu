// Host launchers of the cluster kernel for the bottom of the V-cycle
// (cluster_tail.cuh), in a translation unit of their own.
#include "cluster_tail.cuh"

namespace gmg {

namespace {

template <typename T, int D>
void cluster_attrs(size_t smem, int P) {
  auto kern = k_cycle_cluster<T, D>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  // clusters of 16 CTAs are beyond the portable size of 8
  if (P > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
}

}  // namespace

template <typename T, int D>
cudaError_t launch_cycle_cluster(const GmgView<T> &V, const LvArgs *lvtab, int lmin, const ClusterArgs &A,
                                 int nunits, size_t smem, cudaStream_t s, bool pdl) {
  const int P = D == 3 ? 4 * A.pz : 4;
  cluster_attrs<T, D>(smem, P);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P * nunits);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 2 : 1;
  return cudaLaunchKernelEx(&cfg, k_cycle_cluster<T, D>, V, lvtab, lmin, A);
}

template <typename T, int D>
int cycle_cluster_capacity(size_t smem, int P) {
  cluster_attrs<T, D>(smem, P);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = P;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_cycle_cluster<T, D>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template cudaError_t launch_cycle_cluster<float, 2>(const GmgView<float> &, const LvArgs *, int, const ClusterArgs &,
                                                    int, size_t, cudaStream_t, bool);
template cudaError_t launch_cycle_cluster<float, 3>(const GmgView<float> &, const LvArgs *, int, const ClusterArgs &,
                                                    int, size_t, cudaStream_t, bool);
template cudaError_t launch_cycle_cluster<double, 2>(const GmgView<double> &, const LvArgs *, int,
                                                     const ClusterArgs &, int, size_t, cudaStream_t, bool);
template cudaError_t launch_cycle_cluster<double, 3>(const GmgView<double> &, const LvArgs *, int,
                                                     const ClusterArgs &, int, size_t, cudaStream_t, bool);
template int cycle_cluster_capacity<float, 2>(size_t, int);
template int cycle_cluster_capacity<float, 3>(size_t, int);
template int cycle_cluster_capacity<double, 2>(size_t, int);
template int cycle_cluster_capacity<double, 3>(size_t, int);

}  // namespace gmg

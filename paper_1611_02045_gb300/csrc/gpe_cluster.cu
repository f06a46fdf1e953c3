// gpe_cluster.cu -- instantiations and dispatch of the cluster H phi kernel.
#include "gpe_cluster.cuh"
#include "gpe_csolve.cuh"

namespace gpe {

cudaError_t launch_cluster_apply_H(int is_double, const ClusterHArgs& a, cudaStream_t st) {
  if (is_double) {
    switch (a.M) {
      case 32: return launch_cluster_apply_H_one<double, 32, 8>(a, st);
      case 64: return launch_cluster_apply_H_one<double, 64, 8>(a, st);
      case 128: return launch_cluster_apply_H_one<double, 128, 8>(a, st);
      case 256: return launch_cluster_apply_H_one<double, 256, 8>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.E == 16 && a.rows != 32 && a.M == 256) {
    // single precision, E = 16, 256 x 256 fields with f == phi: the dataflow form
    bool used = false;
    const cudaError_t e = launch_h_batch_flow(a, a.flow_ctr, a.flow_cap, a.status, st, &used);
    if (e != cudaSuccess || used) return e;
  }
  if (a.E == 16) {
    // single precision, E = 16: the streaming (persistent, prefetching) form
    // when the fields are 16-byte aligned, else one field per cluster
    bool ok = false;
    cudaError_t e = cudaSuccess;
    if (a.rows == 32) {
      switch (a.M) {
        case 64: e = launch_cluster_apply_H_stream<float, 64, 16, 32>(a, st, &ok); break;
        case 128: e = launch_cluster_apply_H_stream<float, 128, 16, 32>(a, st, &ok); break;
        case 256: e = launch_cluster_apply_H_stream<float, 256, 16, 32>(a, st, &ok); break;
        default: return cudaErrorInvalidValue;
      }
    } else {
      switch (a.M) {
        case 64: e = launch_cluster_apply_H_stream<float, 64, 16, 16>(a, st, &ok); break;
        case 128: e = launch_cluster_apply_H_stream<float, 128, 16, 16>(a, st, &ok); break;
        case 256: e = launch_cluster_apply_H_stream<float, 256, 16, 16>(a, st, &ok); break;
        default: return cudaErrorInvalidValue;
      }
    }
    if (e != cudaSuccess || ok) return e;
    switch (a.M) {
      case 64: return launch_cluster_apply_H_one<float, 64, 16>(a, st);
      case 128: return launch_cluster_apply_H_one<float, 128, 16>(a, st);
      case 256: return launch_cluster_apply_H_one<float, 256, 16>(a, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.M) {
    case 32: return launch_cluster_apply_H_one<float, 32, 8>(a, st);
    case 64: return launch_cluster_apply_H_one<float, 64, 8>(a, st);
    case 128: return launch_cluster_apply_H_one<float, 128, 8>(a, st);
    case 256: return launch_cluster_apply_H_one<float, 256, 8>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_cluster_solve(int M) {
  switch (M) {
    case 32: return cluster_solve_attrs<32>();
    case 64: return cluster_solve_attrs<64>();
    case 128: return cluster_solve_attrs<128>();
    case 256: return cluster_solve_attrs<256>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cluster_solve(int M, const ClusterSolveArgs& P, cudaStream_t st) {
  switch (M) {
    case 32: return launch_cluster_solve_one<32>(P, st);
    case 64: return launch_cluster_solve_one<64>(P, st);
    case 128: return launch_cluster_solve_one<128>(P, st);
    case 256: return launch_cluster_solve_one<256>(P, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gpe

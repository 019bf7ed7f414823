// Forward kinematics of a serial chain as a parallel prefix product over
// SE(3) (the associative scan that replaces the FK loop for serial chains,
// Sec. III-A), one warp per instance: ^0T_i = T_0 T_1 ... T_i.
//
// Lane l owns bodies 2l and 2l + 1 (chains of up to 64 bodies), forms its
// pair product, and an inclusive Hillis-Steele scan over the 32 lanes
// (5 shuffle steps, each composing with the partial product of the lane d
// below) gives every lane the product up to its pair; the product of the
// lanes below, shifted by one lane, completes the first body of each pair.
// Depth 1 + 5 + 1 compositions instead of the 64 of a sequential loop: a
// latency variant for small batches (the thread-per-instance kernel does
// less work per instance and wins on throughput).
#include "kernels.cuh"

namespace frax {

struct SE3 {
  float R[9];
  V3 p;
};

FD SE3 se3_identity() {
  SE3 t;
#pragma unroll
  for (int k = 0; k < 9; ++k) t.R[k] = (k % 4 == 0) ? 1.f : 0.f;
  t.p = mk(0, 0, 0);
  return t;
}

// a * b = (R_a R_b, p_a + R_a p_b)
FD SE3 se3_mul(const SE3& a, const SE3& b) {
  SE3 c;
  mat_mul(a.R, b.R, c.R);
  c.p = a.p + rot(a.R, b.p);
  return c;
}

__device__ __forceinline__ SE3 se3_shfl_up(const SE3& t, int d) {
  SE3 o;
#pragma unroll
  for (int k = 0; k < 9; ++k) o.R[k] = __shfl_up_sync(0xffffffffu, t.R[k], d);
  o.p.x = __shfl_up_sync(0xffffffffu, t.p.x, d);
  o.p.y = __shfl_up_sync(0xffffffffu, t.p.y, d);
  o.p.z = __shfl_up_sync(0xffffffffu, t.p.z, d);
  return o;
}

// ^parent T_i in internal frames: (R_i Rot_z(q_i), p_i); a free-flyer root:
// its world pose.
template <bool FREE>
__device__ __forceinline__ SE3 joint_tf(const ModelImage<64>& M, int i, const float* q, const Col& col) {
  if (i >= M.nb) return se3_identity();
  if (FREE && i == 0) {
    const RootPose P = root_pose(M, q, col);
    SE3 t;
#pragma unroll
    for (int k = 0; k < 9; ++k) t.R[k] = P.E[k];
    t.p = P.r;
    return t;
  }
  const BodyImage& b = M.body[i];
  float sn, cs;
  joint_sincos(col.in(q, FREE ? i + 6 : i) + b.th0, &sn, &cs);
  SE3 t;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float x = b.R[3 * r], y = b.R[3 * r + 1];  // R Rot_z(q + th0)
    t.R[3 * r] = fmaf(cs, x, sn * y);
    t.R[3 * r + 1] = fmaf(-sn, x, cs * y);
    t.R[3 * r + 2] = b.R[3 * r + 2];
  }
  t.p = mk(b.p[0], b.p[1], b.p[2]);
  return t;
}

__device__ __forceinline__ void pose_out(const ModelImage<64>& M, int i, const SE3& t, float* pose, const Col& col) {
  if (i >= M.nb) return;
  const BodyImage& b = M.body[i];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      col.out(pose, 12 * i + 3 * r + c,
              fmaf(t.R[3 * r], b.Q[3 * c], fmaf(t.R[3 * r + 1], b.Q[3 * c + 1], t.R[3 * r + 2] * b.Q[3 * c + 2])));
  col.out(pose, 12 * i + 9, t.p.x);
  col.out(pose, 12 * i + 10, t.p.y);
  col.out(pose, 12 * i + 11, t.p.z);
}

template <bool FREE>
__global__ void __launch_bounds__(kBlock) k_fk_scan(const __grid_constant__ ModelImage<64> M, int64_t B, int64_t ld,
                                                     const float* q, float* pose) {
  const int lane = threadIdx.x & 31;
  const int64_t b = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (b >= B) return;  // b is uniform across the warp: all 32 lanes stay or leave together
  const Col col{ld, b};
  const int i0 = 2 * lane, i1 = i0 + 1;
  const SE3 T0 = joint_tf<FREE>(M, i0, q, col);
  SE3 P = se3_mul(T0, joint_tf<FREE>(M, i1, q, col));
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const SE3 X = se3_shfl_up(P, d);
    if (lane >= d) P = se3_mul(X, P);
  }
  SE3 E = se3_shfl_up(P, 1);
  if (lane == 0) E = se3_identity();
  pose_out(M, i0, se3_mul(E, T0), pose, col);
  pose_out(M, i1, P, pose, col);
}

cudaError_t launch_fk_scan(const HostModel& m, const OpArgs& a) {
  const ModelImage<64>& img = m.image<64>();
  const int64_t threads = a.B * 32;
  const dim3 grid(unsigned((threads + kBlock - 1) / kBlock));
  if (m.free_root)
    k_fk_scan<true><<<grid, kBlock, 0, a.stream>>>(img, a.B, a.ld, a.q, a.out0);
  else
    k_fk_scan<false><<<grid, kBlock, 0, a.stream>>>(img, a.B, a.ld, a.q, a.out0);
  return cudaGetLastError();
}

}  // namespace frax

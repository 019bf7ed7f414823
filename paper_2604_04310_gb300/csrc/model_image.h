// FP32 model image passed to every kernel by value (__grid_constant__), so
// each launch carries the model in its constant bank and no device memory is
// allocated for it. Shared by the host packer (model.cpp) and the kernels.
#pragma once
#include <stdint.h>

namespace frax {

constexpr int kMaxBodies = 64;
constexpr int kMaxDofs = kMaxBodies + 5;

// One body in its *internal* frame: the user's body frame rotated by a
// constant Q_i chosen so that the revolute joint axis becomes local z.
// Then ^parent'R_i' = R * Rot_z(q_i), the motion subspace is e_z, and
// tau_i is the z component of the body's joint moment.
struct BodyImage {
  float R[9];  // constant rotation child' -> parent' (row-major); for a free
               // root: the placement rotation
  float p[3];  // joint origin in parent' coordinates; free root: placement p
  float Q[9];  // internal -> user body-frame rotation (row-major), for poses
  float m;     // mass
  float h[3];  // first moment m*c in internal coordinates
  float I[6];  // rotational inertia about the body origin, internal coords:
               // xx, yy, zz, xy, xz, yz
};

template <int NB>
struct alignas(16) ModelImage {
  int32_t nb, nq, nv, free_root;
  float g[3];                       // world gravity
  int8_t parent[NB];                // parent body, -1 = world
  int8_t dparent[NB + 5];           // per dof: previous dof towards the root
  uint64_t anc[NB];                 // bit j set iff j in Anc(i) (i included)
  BodyImage body[NB];
};

}  // namespace frax

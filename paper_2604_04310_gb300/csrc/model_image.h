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
// Then ^parent'R_i' = R * Rot_z(q_i + th0), the motion subspace is e_z, and
// tau_i is the z component of the body's joint moment.
//
// The rotation of an internal frame about its own z is free. A body with a
// single (revolute) child turns its x onto the common normal of its axis and
// the child's (the Denavit-Hartenberg choice); the child's R is then a
// rotation about x alone, R = Rot_x(alpha), and the rest of the relative
// rotation, Rot_z(th0), joins the joint angle. Kernels transform through
// such a body with the sparse form (dh != 0): a third of the flops of a
// general R.
struct BodyImage {
  float R[9];  // constant rotation child' -> parent' (row-major); for a free
               // root: the placement rotation
  float p[3];  // joint origin in parent' coordinates; free root: placement p
  float Q[9];  // internal -> user body-frame rotation (row-major), for poses
  float m;     // mass
  float h[3];  // first moment m*c in internal coordinates
  float I[6];  // rotational inertia about the body origin, internal coords:
               // xx, yy, zz, xy, xz, yz
  float ca, sa;  // cos, sin of alpha when R = Rot_x(alpha)
  float th0;     // joint angle offset (0 unless dh)
  int32_t dh;    // R is Rot_x(alpha)
};

// Segments: maximal runs of bodies in which every body but the last has
// exactly one child, the next body of the run (at most kMaxSeg bodies; a
// free-flyer root is a segment of its own). Kernels unroll a segment so its
// per-body state stays in registers. Segments are numbered in topological
// order; `act` lists them depth-first: a leaf segment runs its outward and
// inward sweeps back to back, a segment with child segments runs its outward
// sweep, then its children, then its inward sweep.
constexpr int kMaxSeg = 8;
enum SegAction { kActLeaf = 0, kActOpen = 1, kActClose = 2 };

template <int NB>
struct alignas(16) ModelImage {
  int32_t nb, nq, nv, free_root;
  float g[3];                       // world gravity
  int32_t n_seg, n_act;
  int8_t parent[NB];                // parent body, -1 = world
  int8_t dparent[NB + 5];           // per dof: previous dof towards the root
  int8_t order[NB];                 // bodies grouped by segment
  int8_t seg_start[NB];             // first slot of segment s in `order`
  int8_t seg_len[NB];               // bodies in segment s
  int8_t seg_parent[NB];            // parent body of the segment's first body
  int8_t seg_of[NB];                // segment of body i
  int8_t pos_of[NB];                // slot of body i within its segment
  uint8_t act[2 * NB];              // (action << 6) | segment
  uint64_t anc[NB];                 // bit j set iff j in Anc(i) (i included)
  BodyImage body[NB];
};

// Lane-group schedule: one instance spread over kLgLanes lanes of a warp,
// each lane walking its own root-to-leaf paths of the tree (a heavy-path
// decomposition). An outward sweep runs steps t = 0 .. T-1, lane l handling
// body[t][l] (or idling), all lanes in lockstep; an inward sweep runs the
// same table backwards, so a parent always comes after its children. State
// crosses lanes only where a path starts: the parent's outward state sits in
// its outward slot, a path head's inward contribution in its inward slot.
constexpr int kLgLanes = 4;
enum LgFlag {
  kLgLoad = 1,      // outward: the parent's state comes from its outward slot
  kLgStoreOut = 2,  // outward: this body's state goes to its outward slot
  kLgCarry = 4,     // inward: the lane's carried contribution is a child's
  kLgStoreIn = 8,   // inward: this body's contribution goes to its inward slot
};
struct LanePlan {
  int32_t T;                         // steps of one sweep (0: no plan)
  int32_t n_oslot, n_islot;          // slots used
  int8_t body[kMaxBodies][kLgLanes];  // body at (step, lane), -1 idle
  uint8_t flag[kMaxBodies][kLgLanes];
  int8_t oslot[kMaxBodies];          // per body: outward slot, -1 none
  int8_t islot[kMaxBodies];          // per body: inward slot, -1 none
  int8_t rc_first[kMaxBodies];       // per body: its children whose contributions
  int8_t rc_count[kMaxBodies];       //   sit in inward slots, rc_list[first ..]
  int8_t rc_list[kMaxBodies];
};

}  // namespace frax

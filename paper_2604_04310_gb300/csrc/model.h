// Host-side model: validated FP64 description, derived tree structure, and
// the packed FP32 image the kernels receive.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "model_image.h"

namespace frax {

enum ModelKind { kKindChain = 0, kKindTree = 1 };

struct HostModel {
  int nb = 0, nq = 0, nv = 0;
  bool free_root = false;
  int kind = kKindTree;
  std::vector<int> parent;       // per body
  std::vector<int> iq, iv;       // per body offsets into q / qd
  std::vector<int> dof_parent;   // per dof: previous dof on the path to the root
  std::vector<uint64_t> anc;     // per body ancestor bit mask (self included)
  std::vector<int> depth;        // per body, root = 0
  double gravity[3] = {0, 0, 0};
  std::vector<BodyImage> bodies;  // FP32 internal-frame image

  template <int NB>
  void pack(ModelImage<NB>* img) const;
};

// Validates and derives everything; returns "" on success, else a message.
std::string build_model(int n, const int32_t* parent, const int32_t* joint_type, const double* axis,
                        const double* placement, const double* inertia, const double* gravity,
                        HostModel* out);

template <int NB>
void HostModel::pack(ModelImage<NB>* img) const {
  img->nb = nb;
  img->nq = nq;
  img->nv = nv;
  img->free_root = free_root ? 1 : 0;
  for (int k = 0; k < 3; ++k) img->g[k] = static_cast<float>(gravity[k]);
  for (int i = NB; i < NB + 5; ++i)
    img->dparent[i] = static_cast<int8_t>(i < nv ? dof_parent[i] : -1);
  for (int i = 0; i < NB; ++i) {
    img->parent[i] = static_cast<int8_t>(i < nb ? parent[i] : -1);
    img->anc[i] = i < nb ? anc[i] : 0;
    img->dparent[i] = static_cast<int8_t>(i < nv ? dof_parent[i] : -1);
    if (i < nb) img->body[i] = bodies[i];
    else img->body[i] = BodyImage{};
  }
}

}  // namespace frax

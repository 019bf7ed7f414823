// Host-side model: validated FP64 description, derived tree structure, and
// the packed FP32 image the kernels receive.
#pragma once
#include <stdint.h>

#include <memory>
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
  std::vector<int> order, seg_start, seg_len, seg_parent, act;  // segment schedule
  std::vector<int> seg_of, pos_of;
  std::vector<int> dof_body;        // per dof: its body
  std::vector<uint16_t> zero_M;     // structural zeros of M (entry r * nv + c)
  std::vector<uint16_t> zero_LD;    // and of the packed factor (r (r + 1) / 2 + c)
  double gravity[3] = {0, 0, 0};
  std::vector<BodyImage> bodies;  // FP32 internal-frame image
  LanePlan lane_plan{};            // lockstep lane schedule (model_image.h)

  template <int NB>
  void pack(ModelImage<NB>* img) const;

  // The packed images the batched kernels receive, made once by
  // build_model so a call only copies them into its launch: the chain's
  // (7 and 8 body slots) for 7-body chains, the 32-slot image for trees of
  // up to 32 bodies, and the 64-slot image for every model.
  std::shared_ptr<const ModelImage<7>> img7;
  std::shared_ptr<const ModelImage<8>> img8;
  std::shared_ptr<const ModelImage<32>> img32;
  std::shared_ptr<const ModelImage<64>> img64;
  template <int NB>
  const ModelImage<NB>& image() const;
};

template <>
inline const ModelImage<7>& HostModel::image<7>() const { return *img7; }
template <>
inline const ModelImage<8>& HostModel::image<8>() const { return *img8; }
template <>
inline const ModelImage<32>& HostModel::image<32>() const { return *img32; }
template <>
inline const ModelImage<64>& HostModel::image<64>() const { return *img64; }

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
  img->n_seg = static_cast<int32_t>(seg_start.size());
  img->n_act = static_cast<int32_t>(act.size());
  for (int i = 0; i < NB; ++i) {
    img->order[i] = static_cast<int8_t>(i < nb ? order[i] : 0);
    const bool has = i < img->n_seg;
    img->seg_start[i] = static_cast<int8_t>(has ? seg_start[i] : 0);
    img->seg_len[i] = static_cast<int8_t>(has ? seg_len[i] : 0);
    img->seg_parent[i] = static_cast<int8_t>(has ? seg_parent[i] : -1);
  }
  for (int i = 0; i < NB; ++i) {
    img->seg_of[i] = static_cast<int8_t>(i < nb ? seg_of[i] : 0);
    img->pos_of[i] = static_cast<int8_t>(i < nb ? pos_of[i] : 0);
  }
  for (int i = 0; i < 2 * NB; ++i) img->act[i] = static_cast<uint8_t>(i < img->n_act ? act[i] : 0);
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

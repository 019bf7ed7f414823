// Internal: opaque handle layouts and the thread-local error string shared
// by the C ABI translation units.
#pragma once
#include <string>

#include "../../include/frax.h"
#include <memory>

#include "launch.h"
#include "model.h"

struct frax_model_s {
  frax::HostModel m;
  // Trees: the structural zeros the CRBA kernel writes, per requested output
  // (index 1: M only, 2: the factor only, 3: both), listed once at creation.
  std::unique_ptr<frax::ZeroRows> crba_zeros[4];
  int tree_path = 0;  // FRAX_TREE_PATH_*: how tree kernels spread an instance over threads
};

namespace frax {
frax_status set_error(frax_status s, const std::string& msg);  // returns s
frax_status clear_error();                                      // returns FRAX_OK
}  // namespace frax

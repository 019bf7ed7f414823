// Internal: opaque handle layouts and the thread-local error string shared
// by the C ABI translation units.
#pragma once
#include <string>

#include "../../include/frax.h"
#include "model.h"

struct frax_model_s {
  frax::HostModel m;
};

namespace frax {
frax_status set_error(frax_status s, const std::string& msg);  // returns s
frax_status clear_error();                                      // returns FRAX_OK
}  // namespace frax

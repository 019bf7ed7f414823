// Host-side fault injection for the tests of the server's error paths. A
// test arms one injection point with frax_debug_inject_fault; the next
// `after`-th pass through that point then behaves as if its host allocation
// or CUDA call had failed (the call itself is skipped), once. Nothing is
// injected on the device. Arming is refused unless the process started with
// FRAX_FAULT_INJECTION=1 in its environment, so a production process cannot
// arm it by accident.
#pragma once

namespace frax {

enum FaultPoint {
  kFaultNone = 0,
  kFaultServerAlloc = 1,       // frax_server_create: the server's host struct
  kFaultSlabHost = 2,          // frax_server_create: the pinned host mirror of the slab
  kFaultSubmitInputCopy = 3,   // frax_server_submit: the input copy to the slab
  kFaultSubmitPublish = 4,     // frax_server_submit: the descriptor copy
  kFaultCollectCopy = 5,       // frax_server_collect: the output copy back
  kFaultCount
};

// True when an armed injection fires at `point` (then disarmed).
bool fault_hit(int point);

}  // namespace frax

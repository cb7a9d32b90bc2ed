// Bits of the per-stream device status word (shared by host and device code).
#pragma once

namespace tdp {
enum : unsigned { ST_SINGULAR = 1u, ST_TIMEOUT = 2u, ST_BADARG = 4u };
}  // namespace tdp

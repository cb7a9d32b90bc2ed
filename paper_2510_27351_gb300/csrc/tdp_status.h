// Bits of the per-stream device status word (shared by host and device code).
#pragma once

namespace tdp {
// ST_FALLBACK is informational: the windowed binary32 pass met a tile that
// failed its checks, and the exact binary64 solve produced the answer.
enum : unsigned { ST_SINGULAR = 1u, ST_TIMEOUT = 2u, ST_BADARG = 4u, ST_FALLBACK = 8u };
}  // namespace tdp

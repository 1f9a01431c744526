// Guard-zone bounds checking of the DGT_DEBUG build.
//
// Built with -DDGT_DEBUG (libdgt_debug.so), every device allocation of the library carries a
// guard zone of kGuard bytes on each side, and the workspace of an analysis or synthesis call
// carries one between its regions (Zak transform, Y, the frequency-shear scratch), all filled
// with 0xFF bytes (a NaN in float32 and float64).  After every kernel launch a check kernel
// reads every registered zone on the launching stream; a word that is no longer 0xFFFFFFFF
// counts as a violation (an out-of-bounds write by that launch or an earlier one), is put
// back, and the first one since the last dgt_debug_status call is recorded with the name of
// the launch in a host-mapped word -- nothing traps, the context stays usable.  An
// out-of-bounds read of a guard zone loads NaNs, which the parity comparisons then see.
//
// The debug build serialises its calls (one analysis / synthesis at a time, the device
// synchronised at the end of each) and does not support stream capture; the release build
// compiles all of this away (kDebug false, empty scopes).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace dgt {

constexpr size_t kGuard = 4096;   // bytes of one guard zone (a multiple of 256: alignment is kept)
#ifdef DGT_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif

// device allocation with guard zones on both sides (debug build; plain cudaMalloc otherwise)
cudaError_t dbg_malloc(void** p, size_t bytes);
void dbg_free(void* p);

// after a launch on st: check every registered zone (debug build; nothing otherwise)
void dbg_after_launch(const char* name, cudaStream_t st);

// overwrite the first word of the trailing guard zone of a dbg_malloc allocation of `bytes`
// bytes (inside that allocation), so that the next check reports it; DGT_ERR_UNSUPPORTED in
// the release build
int dbg_touch_trailing_guard(void* p, size_t bytes);

// zones inside a caller's or the plan's workspace, registered for the duration of one call:
// filled on st (and waited for) at construction; at destruction the device is synchronised
// and the zones are dropped.  Empty in the release build.
class DbgScope {
  public:
    DbgScope(cudaStream_t st, char* base, const size_t* offsets, int n);
    ~DbgScope();
    DbgScope(const DbgScope&) = delete;
    DbgScope& operator=(const DbgScope&) = delete;

  private:
    unsigned long long tag_ = 0;
};

}  // namespace dgt

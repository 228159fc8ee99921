// xe_host.h -- host runtime functions shared between translation units (no kernel
// includes this header).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace xe {

// Free the scratch memory the library keeps for stream `s` (staged planes, workspace,
// counters, status word, timing events) once the caller is done with the stream: it waits
// for the stream's work, and a later call on a stream with the same handle starts afresh.
// Used by the streaming server when it closes its compute stream.  Returns an XE_* code.
int release_stream_scratch(cudaStream_t s);

// Size the scratch of stream `s` now for launch groups of up to `max_jobs` jobs of one
// channel each, N inputs and at most `max_T` samples (staged planes, tile counters and the
// split-tile workspace), so that no such batch has to regrow it later: a regrowth
// synchronises the device.  Returns an XE_* code; a buffer that could not be allocated is
// left empty and is allocated by the first batch that needs it.
int reserve_stream_scratch(cudaStream_t s, int max_jobs, int N, int64_t max_T);

// Samples one f32 tensor-memory accumulation may sum (option "exact_chunk_t").
int64_t option_exact_chunk_t();

// The "inject_stall" test hook: returns it and clears it (it applies to one call only).
int take_inject_stall();

}  // namespace xe

// xe_host.h -- host runtime functions shared between translation units (no kernel
// includes this header).
#pragma once
#include <cuda_runtime.h>

namespace xe {

// Free the scratch memory the library keeps for stream `s` (staged planes, workspace,
// counters, status word, timing events) once the caller is done with the stream: it waits
// for the stream's work, and a later call on a stream with the same handle starts afresh.
// Used by the streaming server when it closes its compute stream.  Returns an XE_* code.
int release_stream_scratch(cudaStream_t s);

}  // namespace xe

// Error reporting shared by the translation units of the library (internal header).
#pragma once

namespace fps {

// Record `msg` as the calling thread's last error message without allocating:
// only the pointer is stored, so `msg` must be a string literal (or otherwise
// live for the rest of the process).  fps_last_error() returns it until the next
// failure of any entry point on this thread.
void set_static_error(const char *msg);

}  // namespace fps

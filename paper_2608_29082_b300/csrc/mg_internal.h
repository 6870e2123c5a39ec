// Internal helpers shared by the host translation units of libmg.so.
#pragma once

#include <mutex>
#include <string>

#include "mg.h"

namespace mgi {

// Serialises the host-side work that creates or destroys device state or
// records CUDA graphs (context set-up and destruction, graph capture and
// instantiation) across threads: a context created on one thread while
// another thread records a graph must not meet that capture half-way.
// Graph launches and kernel work are not serialised.  Recursive: set-up
// helpers nest.
std::recursive_mutex& setup_mutex();

// Records a message for calls that have no context (set-up helpers, a failed
// mg_setup) and returns the status unchanged.
mg_status set_global_error(mg_status s, const std::string& msg);
const std::string& global_error();

}  // namespace mgi

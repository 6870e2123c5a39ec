// Internal helpers shared by the host translation units of libmg.so.
#pragma once

#include <string>

#include "mg.h"

namespace mgi {

// Records a message for calls that have no context (set-up helpers, a failed
// mg_setup) and returns the status unchanged.
mg_status set_global_error(mg_status s, const std::string& msg);
const std::string& global_error();

}  // namespace mgi

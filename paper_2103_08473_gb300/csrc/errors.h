// Error text of calls made without a context (read back with ccsd_last_error(NULL)).
#pragma once

#include <string>

namespace ccsd {
void set_context_free_error(const std::string& msg);
}  // namespace ccsd

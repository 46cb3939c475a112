// Library-internal declarations shared by the translation units of libfsi.so
// (not part of the C ABI).
#pragma once
#include <string>

// Sets the calling thread's fsi_last_error() message and returns code.
int fsi_record_error(int code, const std::string& msg);

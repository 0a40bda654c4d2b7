// Shared between the host entry points (capi.cpp) and the device executor (exec.cu).
#pragma once

#include <exception>
#include <map>
#include <memory>
#include <new>
#include <string>

#include "../../include/tnc.h"
#include "host.h"

namespace tnc {

void set_error(const std::string& m);

// Runs `f`, mapping exceptions to status codes and the thread-local message.
template <class F>
tnc_status guarded(F&& f) {
  try {
    f();
    set_error("");
    return TNC_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return TNC_E_OOM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return TNC_E_INVALID_ARG;
  } catch (...) {
    set_error("unknown error");
    return TNC_E_INVALID_ARG;
  }
}

struct DeviceProgram;  // defined in exec.cu

}  // namespace tnc

struct tnc_plan_s {
  tnc::Plan p;
  // device programs compiled for this plan, keyed by (context id, precision, wave, fuse)
  std::map<std::string, std::shared_ptr<tnc::DeviceProgram>> programs;
};

namespace tnc {
void release_plan_device(tnc_plan_s* p);
}

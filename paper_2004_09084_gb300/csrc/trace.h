// Optional NVTX ranges around the library's host calls.  A decode is one
// persistent launch that runs every layer group of every iteration, so a host
// range covers the whole launch; its name states the layer-group schedule
// (groups per iteration x iterations) and the kernel, and qcmet_decode_host
// nests ranges for its copies.  Off unless the environment variable
// QCMET_NVTX is set to 1 when the library is first used; without a tool
// attached the NVTX calls cost next to nothing either way.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace qcmet {

inline bool nvtx_enabled() {
    static const bool on = [] {
        const char *v = std::getenv("QCMET_NVTX");
        return v && std::strcmp(v, "1") == 0;
    }();
    return on;
}

// A scoped range in the "qcmet" domain; the name is formatted printf-style.
class TraceRange {
  public:
    template <typename... A>
    explicit TraceRange(const char *fmt, A... args) {
        if (!nvtx_enabled()) return;
        char name[160];
        std::snprintf(name, sizeof name, fmt, args...);
        nvtxEventAttributes_t at = {};
        at.version = NVTX_VERSION;
        at.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        at.messageType = NVTX_MESSAGE_TYPE_ASCII;
        at.message.ascii = name;
        nvtxDomainRangePushEx(domain(), &at);
        active_ = true;
    }
    ~TraceRange() {
        if (active_) nvtxDomainRangePop(domain());
    }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;

  private:
    static nvtxDomainHandle_t domain() {
        static nvtxDomainHandle_t d = nvtxDomainCreateA("qcmet");
        return d;
    }
    bool active_ = false;
};

}  // namespace qcmet

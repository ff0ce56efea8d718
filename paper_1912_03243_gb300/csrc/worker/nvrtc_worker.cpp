// Compile worker for the tiled pass kernels.  NVRTC serialises compilations
// inside one process, so the library runs several of these at once, one per
// pass, and loads the cubins they write.
//
//   sv_nvrtc_worker <source file> <cubin file> <verbose: 0 | 1>
//
// Exit status 0 with the cubin written; 1 with NVRTC's log on stderr (the
// log also goes to stderr when verbose); 2 for bad arguments or files.
#include <nvrtc.h>

#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>

#include "../nvrtc_opts.h"

int main(int argc, char **argv) {
    if (argc != 4) {
        std::fprintf(stderr, "usage: %s <source> <cubin> <verbose 0|1>\n", argc > 0 ? argv[0] : "sv_nvrtc_worker");
        return 2;
    }
    std::ifstream in(argv[1], std::ios::binary);
    if (!in) {
        std::fprintf(stderr, "cannot read %s\n", argv[1]);
        return 2;
    }
    std::stringstream ss;
    ss << in.rdbuf();
    const std::string src = ss.str();
    const bool verbose = argv[3][0] == '1';
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "sv_pass.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        std::fprintf(stderr, "nvrtcCreateProgram failed\n");
        return 1;
    }
    const nvrtcResult r =
        nvrtcCompileProgram(prog, verbose ? sv::kPassNvrtcOptsVerbose : sv::kPassNvrtcOptsQuiet, sv::kPassNvrtcOpts);
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    if (r != NVRTC_SUCCESS || verbose) std::fprintf(stderr, "%s\n", log.c_str());
    if (r != NVRTC_SUCCESS) {
        std::fprintf(stderr, "%s\n", nvrtcGetErrorString(r));
        nvrtcDestroyProgram(&prog);
        return 1;
    }
    size_t cs = 0;
    nvrtcGetCUBINSize(prog, &cs);
    std::string cubin(cs, '\0');
    nvrtcGetCUBIN(prog, &cubin[0]);
    nvrtcDestroyProgram(&prog);
    std::ofstream out(argv[2], std::ios::binary);
    out.write(cubin.data(), std::streamsize(cubin.size()));
    out.close();
    return out ? 0 : 2;
}

// tune.cu — the autotuner's cache: tuned plan options kept in a JSON file,
// keyed by the GPU (name and SM count) and the plan's signature, so that a
// tuned shape is timed once per machine and later plans reuse the choice.
//
// File format (written by this file, read tolerantly):
//   {"version": 1, "entries": {"<gpu>|<sms>|<signature>": {"<option>": <number>, ...}, ...}}
// Path: $GBFFT_TUNE_CACHE if set (empty = no cache), else
// $XDG_CACHE_HOME/gbfft/tune.json or $HOME/.cache/gbfft/tune.json.  Writes go
// to a temporary file renamed over the old one, so readers never see a
// half-written file; concurrent writers may lose each other's entries (the
// cost is a re-tune, never a wrong choice, since every entry is complete).
#include <cuda_runtime.h>
#include <sys/stat.h>
#include <unistd.h>

#include <cctype>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>

#include "tune.h"

namespace gbfft {

namespace {

// minimal recursive-descent reader for the subset written below: objects,
// strings (with \" and \\ escapes), numbers; anything else fails the parse
struct Reader {
    const std::string &s;
    size_t i = 0;
    explicit Reader(const std::string &t) : s(t) {}
    void ws() {
        while (i < s.size() && isspace((unsigned char)s[i])) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < s.size() && s[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    bool str(std::string &out) {
        ws();
        if (i >= s.size() || s[i] != '"') return false;
        ++i;
        out.clear();
        while (i < s.size() && s[i] != '"') {
            if (s[i] == '\\' && i + 1 < s.size()) ++i;
            out.push_back(s[i++]);
        }
        if (i >= s.size()) return false;
        ++i;
        return true;
    }
    bool num(double &v) {
        ws();
        const char *b = s.c_str() + i;
        char *e = nullptr;
        v = strtod(b, &e);
        if (e == b) return false;
        i += (size_t)(e - b);
        return true;
    }
    bool entry(TuneEntry &out) {  // {"k": number, ...}
        if (!eat('{')) return false;
        if (eat('}')) return true;
        do {
            std::string k;
            double v;
            if (!str(k) || !eat(':') || !num(v)) return false;
            out[k] = v;
        } while (eat(','));
        return eat('}');
    }
};

std::string quote(const std::string &k) {
    std::string o = "\"";
    for (char c : k) {
        if (c == '"' || c == '\\') o.push_back('\\');
        o.push_back(c);
    }
    return o + "\"";
}

void make_dirs(const std::string &path) {
    for (size_t p = path.find('/', 1); p != std::string::npos; p = path.find('/', p + 1))
        mkdir(path.substr(0, p).c_str(), 0755);
}

}  // namespace

std::string tune_cache_path() {
    if (const char *e = getenv("GBFFT_TUNE_CACHE")) return std::string(e);
    if (const char *x = getenv("XDG_CACHE_HOME"); x && *x) return std::string(x) + "/gbfft/tune.json";
    if (const char *h = getenv("HOME"); h && *h) return std::string(h) + "/.cache/gbfft/tune.json";
    return std::string();
}

std::string tune_device_key() {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        cudaGetLastError();
        return std::string("unknown|0");
    }
    std::ostringstream o;
    o << prop.name << "|" << prop.multiProcessorCount;
    return o.str();
}

bool tune_cache_load(const std::string &path, TuneCache &out) {
    out.clear();
    if (path.empty()) return false;
    std::ifstream f(path);
    if (!f) return false;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string text = ss.str();
    Reader r(text);
    if (!r.eat('{')) return false;
    do {
        std::string k;
        if (!r.str(k) || !r.eat(':')) return false;
        if (k == "entries") {
            if (!r.eat('{')) return false;
            if (!r.eat('}')) {
                do {
                    std::string key;
                    TuneEntry e;
                    if (!r.str(key) || !r.eat(':') || !r.entry(e)) return false;
                    out[key] = e;
                } while (r.eat(','));
                if (!r.eat('}')) return false;
            }
        } else {
            double v;
            if (!r.num(v)) return false;
        }
    } while (r.eat(','));
    return r.eat('}');
}

bool tune_cache_store(const std::string &path, const TuneCache &in) {
    if (path.empty()) return false;
    make_dirs(path);
    std::ostringstream o;
    o << "{\"version\": 1, \"entries\": {";
    bool first = true;
    for (const auto &kv : in) {
        o << (first ? "\n  " : ",\n  ") << quote(kv.first) << ": {";
        first = false;
        bool f2 = true;
        for (const auto &ov : kv.second) {
            char buf[64];
            snprintf(buf, sizeof buf, "%.6g", ov.second);
            o << (f2 ? "" : ", ") << quote(ov.first) << ": " << buf;
            f2 = false;
        }
        o << "}";
    }
    o << "\n}}\n";
    const std::string tmp = path + ".tmp" + std::to_string((long long)getpid());
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return false;
        f << o.str();
        if (!f) return false;
    }
    if (rename(tmp.c_str(), path.c_str()) != 0) {
        unlink(tmp.c_str());
        return false;
    }
    return true;
}

}  // namespace gbfft

// tune.h — the autotuner's cache of tuned plan options (tune.cu).  Not installed.
#pragma once

#include <map>
#include <string>

namespace gbfft {

typedef std::map<std::string, double> TuneEntry;      // option name -> value (and measured times)
typedef std::map<std::string, TuneEntry> TuneCache;   // "<gpu>|<sms>|<signature>" -> entry

std::string tune_cache_path();   // "" = no cache
std::string tune_device_key();   // "<gpu name>|<SM count>" of the current device
bool tune_cache_load(const std::string &path, TuneCache &out);
bool tune_cache_store(const std::string &path, const TuneCache &in);

}  // namespace gbfft

"""The autotuner's cache file (csrc/tune_cache.h, host-only C++): round trips
of keys with quotes, backslashes and spaces, several keys in one file,
overwrites, and tolerance of missing or malformed files; and the argument
checks of the chunk and autotune entry points that need no device.  CPU
only."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

DRIVER = r"""
#include <cstdio>
#include <string>
#include "tune_cache.h"
// usage: get PATH KEY | put PATH KEY VALUE | parse PATH
int main(int argc, char** argv) {
  std::string op = argv[1], path = argv[2];
  if (op == "get") {
    long v = 0;
    if (!nlc::tune_cache_get(path, argv[3], &v)) { std::puts("absent"); return 0; }
    std::printf("%ld\n", v);
    return 0;
  }
  if (op == "put") return nlc::tune_cache_put(path, argv[3], std::stol(argv[4])) ? 0 : 1;
  if (op == "parse") {
    std::map<std::string, long> m;
    FILE* f = std::fopen(path.c_str(), "rb");
    std::string t;
    char b[256];
    size_t k;
    while (f && (k = std::fread(b, 1, sizeof b, f)) > 0) t.append(b, k);
    if (f) std::fclose(f);
    const bool ok = nlc::tune_cache_parse(t, &m);
    std::printf("%d %zu\n", ok ? 1 : 0, m.size());
    return 0;
  }
  return 2;
}
"""


@pytest.fixture(scope="module")
def tool(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("tc")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    exe = d / "drv"
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-I",
                           os.path.join(ROOT, "paper_1907_13415_gb300", "csrc"),
                           str(src), "-o", str(exe)])

    def run(*args):
        return subprocess.run([str(exe), *map(str, args)], capture_output=True,
                              text=True)
    return run


def test_round_trip_and_json(tool, tmp_path):
    path = tmp_path / "tune.json"
    keys = {"D3Q19/fp32/n1/256x256x256/std/NVIDIA GB300/152": 16,
            'odd "quoted" \\ key': 7,
            "D2Q9/fp64/n2/64x64x1,32x32x1m/iso/GPU/1": 1}
    assert tool("get", path, "x").stdout.strip() == "absent"  # no file yet
    for k, v in keys.items():
        assert tool("put", path, k, v).returncode == 0
    for k, v in keys.items():
        assert tool("get", path, k).stdout.strip() == str(v)
    # the file is plain JSON with exactly these entries
    assert json.loads(path.read_text()) == keys
    # overwrite keeps the others
    first = next(iter(keys))
    assert tool("put", path, first, 32).returncode == 0
    assert json.loads(path.read_text()) == dict(keys, **{first: 32})
    assert not [p for p in os.listdir(tmp_path) if ".tmp." in p]


def test_malformed_files_read_as_empty(tool, tmp_path):
    path = tmp_path / "bad.json"
    for text in ["", "[1, 2]", '{"a": }', '{"a": 1', '{"a" 1}', "garbage"]:
        path.write_text(text)
        assert tool("get", path, "a").stdout.strip() == "absent", text
        assert tool("parse", path).stdout.split()[1] == "0", text
    path.write_text('{\n  "a": 3,\n  "b": -1\n}\n')
    assert tool("parse", path).stdout.split() == ["1", "2"]
    # a put on a malformed file starts a fresh one
    path.write_text("{broken")
    assert tool("put", path, "k", 4).returncode == 0
    assert json.loads(path.read_text()) == {"k": 4}


def test_unwritable_cache_reports_failure(tool, tmp_path):
    path = tmp_path / "no_such_dir" / "tune.json"
    assert tool("put", path, "k", 1).returncode == 1


def test_chunk_and_autotune_reject_null_context():
    from paper_1907_13415_gb300 import nlc
    lib = nlc.load()
    assert lib.nlc_set_chunk(None, 8, 0) == -1
    assert lib.nlc_get_chunk(None, 0, None) == -1
    assert lib.nlc_autotune(None, 5, None) == -1

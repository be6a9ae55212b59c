"""The CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer:
tests/oracle_sanitize.c drives every entry point of oracle.c with random and
edge-case inputs in buffers of exactly the documented capacity and
cross-checks the independent routes to the same hull.  An out-of-bounds
access, undefined arithmetic, a leak or a disagreement fails the test.  Only
a missing sanitizer runtime skips it."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = [os.path.join(ROOT, "oracle", "oracle.c"), os.path.join(ROOT, "tests", "oracle_sanitize.c")]


def test_oracle_is_clean_under_sanitizers(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    base = [gcc, "-std=gnu11", "-O1", "-g", *SRC, "-lm"]
    plain = subprocess.run(base + ["-o", str(tmp_path / "plain")], capture_output=True, text=True)
    assert plain.returncode == 0, plain.stderr[-2000:]  # a real build error is a failure
    # the cross-checks hold without sanitizers too
    r = subprocess.run([str(tmp_path / "plain"), "5000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "oracle sanitize ok" in r.stdout, r.stderr[-2000:]
    exe = tmp_path / "osan"
    san = subprocess.run(base[:4] + ["-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                                     "-fno-omit-frame-pointer"] + base[4:] + ["-o", str(exe)],
                         capture_output=True, text=True)
    if san.returncode != 0:
        pytest.skip("no sanitizer runtime for gcc here")
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1")
    probe = subprocess.run([str(exe), "0"], capture_output=True, text=True, env=env, timeout=120)
    if probe.returncode != 0 and "LeakSanitizer" in probe.stderr:
        env["ASAN_OPTIONS"] = "detect_leaks=0"  # leak checking unavailable here
        probe = subprocess.run([str(exe), "0"], capture_output=True, text=True, env=env, timeout=120)
    if probe.returncode != 0:
        pytest.skip("the sanitizer runtime cannot run here: " + probe.stderr[-200:])
    r = subprocess.run([str(exe), "20000"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "oracle sanitize ok" in r.stdout


def test_a_planted_overrun_is_reported(tmp_path):
    """The harness can see a mistake: a copy of the oracle whose bit-array
    writer stores one word past its buffer fails the run."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    text = open(SRC[0]).read()
    head = "void oracle_mask(const int32_t *L, int32_t p, uint32_t *M)\n{"
    assert head in text
    planted = tmp_path / "oracle_planted.c"
    planted.write_text(text.replace(head, head + "\n    M[(p + 31) / 32] = 0;", 1))
    exe = tmp_path / "osan_planted"
    san = subprocess.run([gcc, "-std=gnu11", "-O1", "-g", "-fsanitize=address,undefined",
                          "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", str(planted), SRC[1],
                          "-lm", "-o", str(exe)], capture_output=True, text=True)
    if san.returncode != 0:
        pytest.skip("no sanitizer runtime for gcc here")
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0")
    probe = subprocess.run([str(exe), "0"], capture_output=True, text=True, env=env, timeout=120)
    if probe.returncode != 0:  # no trial reaches the planted line
        pytest.skip("the sanitizer runtime cannot run here: " + probe.stderr[-200:])
    r = subprocess.run([str(exe), "50"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode != 0 and "heap-buffer-overflow" in r.stderr

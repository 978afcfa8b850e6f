"""Compile the FP64 CPU oracle (plain C) into a shared library beside this file.

Test infrastructure: the library it builds is the reference the CUDA path is
checked against.  FP contraction is off so every multiply and add rounds
separately, in the order the source states.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbm_oracle.c")
LIB = os.path.join(HERE, "_lbm_oracle.so")
# tuned for the CPU it is built on; built where it runs (the timed CPU baseline),
# never shipped to another machine.  Without FP contraction or reassociation the
# tuning changes speed, not results.
LIB_NATIVE = os.path.join(HERE, "_lbm_oracle_native.so")


def build(force: bool = False, native: bool = False) -> str:
    lib = LIB_NATIVE if native else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(SRC) and \
            (not native or _built_here(lib)):
        return lib
    arch = ["-march=native"] if native else []
    cmd = ["gcc", "-O3", *arch, "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
           "-fPIC", "-shared", "-Wall", "-Wno-unknown-pragmas", "-o", lib + ".tmp", SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)
    if native:
        with open(lib + ".cpu", "w") as fh:
            fh.write(_cpu_id())
    return lib


def _cpu_id():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _built_here(lib):
    try:
        with open(lib + ".cpu") as fh:
            return fh.read() == _cpu_id()
    except OSError:
        return False


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))

"""Compile the oracle's C code into oracle/liboracle.so (test infrastructure)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "usr_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


LIB_SAN = os.path.join(HERE, "liboracle_san.so")


def build(force: bool = False) -> str:
    """Build liboracle.so with gcc (OpenMP, no FP contraction) if it is stale.

    With ORACLE_SANITIZE=1 in the environment, build and return liboracle_san.so instead: the same code
    under AddressSanitizer and UndefinedBehaviorSanitizer (load it with the sanitizer runtimes preloaded,
    e.g. LD_PRELOAD="$(gcc -print-file-name=libasan.so) $(gcc -print-file-name=libubsan.so)").
    """
    san = os.environ.get("ORACLE_SANITIZE") == "1"
    lib = LIB_SAN if san else LIB
    # stale when the source or this file (its flags) is newer than the library
    newest = max(os.path.getmtime(SRC), os.path.getmtime(os.path.abspath(__file__)))
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    tmp = lib + ".tmp%d" % os.getpid()
    flags = ["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined,float-cast-overflow",
             "-fno-sanitize-recover=undefined,float-cast-overflow"] if san else ["-O2"]
    cmd = ["gcc"] + flags + ["-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                             SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))

"""Build libhairfuse.so in-tree with nvcc for sm_103a (B300)."""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libhairfuse.so")

NVCC_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-Xcompiler", "-fPIC",
    "-Xptxas", "-v",
]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def build(verbose=False):
    """Compile every .cu under csrc/ (in parallel, one object each) and link them into one shared
    library; returns its path."""
    from concurrent.futures import ThreadPoolExecutor
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    srcs = sources()
    objs = [os.path.join(objdir, os.path.basename(f)[:-3] + ".o") for f in srcs]

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc, *NVCC_FLAGS, "-c", "-o", obj, src]
        res = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, res

    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 1)) as ex:
        results = list(ex.map(compile_one, zip(srcs, objs)))
    link = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", LIB, *objs]
    lres = subprocess.run(link, capture_output=True, text=True) if all(r.returncode == 0 for _, r in results) else None
    log = "".join(" ".join(c) + "\n" + r.stdout + r.stderr for c, r in results)
    if lres is not None:
        log += " ".join(link) + "\n" + lres.stdout + lres.stderr
    with open(os.path.join(HERE, "build.log"), "w") as f:
        f.write(log)
    if lres is None or lres.returncode != 0:
        sys.stderr.write(log)
        raise RuntimeError("nvcc failed building libhairfuse.so")
    if verbose:
        sys.stdout.write(log)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
    print(LIB)

"""Build the CUDA library libwavepacket_gpu.so in-tree for sm_103a (GB300).

The translation units compile in parallel with nvcc and link into
paper_1306_3247_gb300/_lib/libwavepacket_gpu.so. Nothing is installed elsewhere.
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libwavepacket_gpu.so")
SOURCES = ["wp_api.cu", "wp_kernels_f64.cu", "wp_kernels_f32.cu", "wp_kernels_ff.cu", "wp_fixed_f64.cu",
           "wp_fixed_f32.cu", "wp_fixed_ff.cu", "wp_fixed_obs_f64.cu", "wp_fixed_obs_f32.cu", "wp_fixed_obs_ff.cu",
           "wp_fixed_grid_f64.cu", "wp_fixed_grid_f32.cu", "wp_fixed_grid_ff.cu",
           "wp_batch_f64_contig.cu", "wp_batch_f64_strided.cu", "wp_batch_f32_contig.cu", "wp_batch_f32_strided.cu",
           "wp_batch_ff_contig.cu", "wp_batch_ff_strided.cu", "wp_res1d_f64.cu", "wp_res1d_f32.cu", "wp_res1d_ff.cu",
           "wp_noalloc.cu", "wp_server.cu", "wp_jit.cu", "wp_probe.cu",
           "wp_pass256_f32.cu", "wp_pass256_ff.cu", "wp_pass2s_f32.cu", "wp_batch_merged_f32_contig.cu", "wp_batch_merged_f32_strided.cu",
           "wp_batch_merged_f64_contig.cu", "wp_batch_merged_f64_strided.cu", "wp_batch_merged_ff_contig.cu",
           "wp_batch_merged_ff_strided.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "wavepacket_gpu.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(f"--- {s}\n{o}" for s, o in failed))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))

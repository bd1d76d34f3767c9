"""The C example in README.md compiles against include/pmsp.h, links against the
library and runs: without a GPU it stops at pmsp_create with PMSP_ECUDA (exit 2);
with one it densifies and prints the mean range."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_c_example(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    import torch
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", text, flags=re.S)
    assert len(blocks) == 1
    src = tmp_path / "example.c"
    src.write_text(blocks[0])
    exe = tmp_path / "example"
    libdir = os.path.join(ROOT, "paper_2211_16266_gb300")
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                           str(src), "-L", libdir, "-lpmsp", f"-Wl,-rpath,{libdir}", "-lm"])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    if torch.cuda.is_available():
        assert r.returncode == 0 and r.stdout.startswith("mean range"), r.stderr
    else:
        assert r.returncode == 2 and "pmsp_create: -6" in r.stderr, (r.returncode, r.stderr)

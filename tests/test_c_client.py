"""The C ABI from C: include/etdm.h compiles as strict C99 and a C program
links against libetdm.so and gets the documented answers from the calls that
return before any device work (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c99_client_compiles_links_and_runs(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2101_12597_gb300 import build
    build.build()
    libdir = os.path.join(ROOT, "paper_2101_12597_gb300")
    exe = str(tmp_path / "abi_client")
    subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_client.c"),
                    "-L", libdir, "-letdm", f"-Wl,-rpath,{libdir}", "-pthread", "-o", exe],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    assert len(lines) >= 15 and all(ln.startswith("ok ") for ln in lines), r.stdout


def test_readme_c_example_compiles_and_links(tmp_path):
    """The C example of the README is valid C99 against include/etdm.h and
    links against libetdm.so (it needs a GPU to run, so it is only built)."""
    import re
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2101_12597_gb300 import build
    build.build()
    txt = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```c\n(.*?)```", txt, flags=re.S)
    assert len(blocks) == 1
    src = tmp_path / "readme_example.c"
    src.write_text(blocks[0] + "\nint main(void) { return 0; }\n")
    libdir = os.path.join(ROOT, "paper_2101_12597_gb300")
    subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-letdm", f"-Wl,-rpath,{libdir}",
                    "-o", str(tmp_path / "readme_example")], check=True)

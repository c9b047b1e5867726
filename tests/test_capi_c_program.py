"""include/wmgct.h is a C header: a C99 program that includes it, takes the
address of every call it declares and runs the calls that need no GPU
(version, last error, allocator registration) compiles with -Wall -Werror,
links against libwmgct.so and runs on a machine without a GPU."""
import os
import re
import shutil
import subprocess

import pytest

import paper_1310_0956_gb300 as wmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "include")


def declared():
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(INC, "wmgct.h")).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(wmg_[a-z0-9_]+)\s*\(", src)))


def test_header_compiles_and_links_as_c(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lib = wmg.build()
    names = declared()
    refs = "\n".join(f"    (void *)&{n}," for n in names)
    prog = f"""
#include <stdio.h>
#include <string.h>
#include "wmgct.h"

static void *no_alloc(size_t bytes, void *stream, void *ctx) {{ (void)bytes; (void)stream; (void)ctx; return NULL; }}
static void no_free(void *p, size_t bytes, void *stream, void *ctx) {{ (void)p; (void)bytes; (void)stream; (void)ctx; }}

int main(void) {{
    void *calls[] = {{
{refs}
    }};
    char msg[256];
    size_t i;
    for (i = 0; i < sizeof calls / sizeof calls[0]; ++i)
        if (!calls[i]) return 1;
    if (wmg_version() < 100) return 2;
    if (wmg_set_allocator(no_alloc, NULL, NULL) != WMG_ERR_INVALID_ARG) return 3;
    wmg_last_error(msg, sizeof msg);
    if (strlen(msg) == 0) return 4;
    if (wmg_set_allocator(no_alloc, no_free, NULL) != WMG_OK) return 5;
    if (wmg_set_allocator(NULL, NULL, NULL) != WMG_OK) return 6;
    printf("%d %d\\n", (int)(sizeof calls / sizeof calls[0]), wmg_version());
    return 0;
}}
"""
    src = tmp_path / "use_wmgct.c"
    exe = tmp_path / "use_wmgct"
    src.write_text(prog)
    libdir = os.path.dirname(lib)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", INC, str(src), "-o", str(exe), "-L", libdir, "-lwmgct", f"-Wl,-rpath,{libdir}"],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out
    count, version = map(int, out.stdout.split())
    assert count == len(names) and version >= 100


def test_readme_c_example_compiles(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    readme = open(os.path.join(ROOT, "README.md")).read()
    snippet = re.search(r"```c\n(.*?)```", readme, flags=re.S).group(1)
    lines = [ln for ln in snippet.splitlines() if not ln.startswith("#include")]
    prog = ('#include "wmgct.h"\n'
            "int example(void *stream, const float *d_b, float *d_x) {\n" + "\n".join(lines) +
            "\n    return rc;\n}\n")
    src = tmp_path / "readme_example.c"
    src.write_text(prog)
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-Wno-unused-variable", "-I", INC, "-c", str(src),
                    "-o", str(tmp_path / "readme_example.o")], check=True)

"""The ncu summaries under profiles/ are short text, and every command they give runs
files of this repository only (CPU only)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def _summaries():
    return sorted(f for f in os.listdir(PROF) if f.endswith(".md"))


def test_summaries_are_short_text():
    for f in os.listdir(PROF):
        path = os.path.join(PROF, f)
        assert f.endswith((".md", ".txt", ".json")), f
        assert os.path.getsize(path) < 64 * 1024, f


def test_commands_name_existing_repository_files():
    seen = 0
    for f in _summaries():
        text = open(os.path.join(PROF, f)).read()
        for block in re.findall(r"```(.*?)```", text, flags=re.S):
            cmd = block.replace("\\\n", " ")
            assert "_work" not in cmd, (f, cmd)
            for tok in re.findall(r"[\w./-]+\.py\b", cmd):
                assert os.path.exists(os.path.join(ROOT, tok)), (f, tok)
                seen += 1
    assert seen >= 4


def test_traffic_entries_name_a_translation_unit():
    import json

    import bench

    d = json.load(open(os.path.join(PROF, "ncu_traffic.json")))
    for kernel, entry in d.items():
        assert kernel in bench.KERNEL_UNITS, kernel
        assert set(entry) >= {"source_hash", "dram_bytes_per_launch", "note"}
        assert entry["dram_bytes_per_launch"] > 0


def test_code_hash_ignores_comments_only():
    import bench

    a = 'int f(int x) { return x + 1; }  // one\n/* block\n comment */\nconst char* s = "/* kept */ // kept";\n'
    b = '/* other words */ int f(int x)   { return x + 1; }\n\n\nconst char* s = "/* kept */ // kept"; // two\n'
    c = 'int f(int x) { return x + 2; }\nconst char* s = "/* kept */ // kept";\n'
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)  # code changed
    assert "/* kept */" in bench.code_only(a)
    assert bench.code_only("char q = '\\''; // x") == "char q = '\\'';"  # an escaped quote
    assert bench.code_only("char b = '\\\\'; // x") == "char b = '\\\\';"  # an escaped backslash

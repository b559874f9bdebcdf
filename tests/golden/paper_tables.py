"""Reader of the values the paper prints in Tables 1 and 2 (Sec. 3), stored
as text in paper_tables_1_2.txt next to this file."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    """{(table, problem, quantity): [L1, ..., L5]}"""
    out = {}
    with open(os.path.join(HERE, "paper_tables_1_2.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            out[(line[0], line[1], line[2])] = [int(t) for t in line[3:]]
    return out

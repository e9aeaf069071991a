"""Rasterise the worked example of the near-contact criterion.

Source: Section 2.3, figure "fig:criterion" (two panels).  The figure fills
cell (col, row) of a 20x10 (left) or 10x10 (right) grid when the distance
from (col, row) to a disc centre is below the disc radius; the discs and the
5x5 stencils are the ones the figure draws:

  left : field i discs (4.356, 2.65) r=4 [tag 1] and (15, 6.2) r=3.5 [tag 2];
         field j disc (15.62, 1.5) r=2.5, drawn on top of field i;
         stencil cols 8-12, rows 2-6, centre cell (10, 4).
  right: field i discs (0,2), (7,2), (5,0), (0,9), all r=3.5 (tag 1);
         stencil cols 2-6, rows 3-7, centre cell (4, 5).

The caption states: left, Step 1 and Step 3 both hold (two tags); right,
Step 1 holds and Step 3 does not (a single tag).  This script writes the
cell grids as text ('.' empty, 'i' field i, 'j' field j), row 0 first.
"""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def raster(ncols, nrows, discs):
    return [[any(math.hypot(col - cx, row - cy) < r for cx, cy, r in discs)
             for col in range(ncols)] for row in range(nrows)]


def write(name, grid_i, grid_j=None):
    rows = []
    for r, line in enumerate(grid_i):
        s = ""
        for col, v in enumerate(line):
            if grid_j is not None and grid_j[r][col]:
                s += "j"
            elif v:
                s += "i"
            else:
                s += "."
        rows.append(s)
    with open(os.path.join(HERE, name), "w") as f:
        f.write("\n".join(rows) + "\n")


def main():
    left_i = raster(20, 10, [(4.356, 2.65, 4.0), (15.0, 6.2, 3.5)])
    left_j = raster(20, 10, [(15.62, 1.5, 2.5)])
    write("criterion_left.txt", left_i, left_j)
    right_i = raster(10, 10, [(0, 2, 3.5), (7, 2, 3.5), (5, 0, 3.5), (0, 9, 3.5)])
    write("criterion_right.txt", right_i)


if __name__ == "__main__":
    main()

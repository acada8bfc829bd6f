"""CPU oracle of the source-box types of Alg. 6 (Sec. 3.2).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``).

For node J of a partition of the space at level l_par (each source box of
that level owned by one node), Alg. 6 sorts every source box of levels 2..L
into DOMESTIC, EXPORT, IMPORT, ROOT and OTHERS, with the critical level
l_crit = max(l_par - 1, 2).  The printed algorithm needs readings (the same
as the library's):

  * "on J": a box of level >= l_par is on J when its ancestor at l_par (the
    box itself at l_par) is owned by J; a box of level <= l_par has children
    on J / off J when some descendant at l_par is owned / not owned by J (the
    algorithm writes "children at l_crit" in one place; ownership is defined
    at l_par, so that is where it is read);
  * M2L neighbours of a source box: the source boxes of its E4 list in the
    source tree (the relation is symmetric);
  * the final assignment after the barrier keeps the marks other boxes' threads
    wrote (as printed it would overwrite them): a box that is not on J is
    IMPORT when some box on J has it as an M2L neighbour, else OTHERS; at
    l_crit a box with no child on J is IMPORT, one with children on and off J
    is ROOT.

Step by step for a box k at level l (the algorithm's flags):
  l < l_crit:  DOMESTIC.
  l = l_crit:  isOnNode = some child on J; isImportExport = some child off J;
               not isOnNode -> IMPORT; isImportExport -> ROOT;
               isExport = some M2L neighbour has a child off J -> EXPORT;
               else DOMESTIC.
  l > l_crit:  k not on J -> IMPORT if some M2L neighbour is on J, else OTHERS;
               k on J: isExport = some M2L neighbour not on J -> EXPORT,
               else DOMESTIC.
"""
from __future__ import annotations

import numpy as np

DOMESTIC, EXPORT, IMPORT, ROOT, OTHERS = 0, 1, 2, 3, 4


def box_types(tree: dict, lpar: int, owner, node: int) -> dict:
    """Types (uint8, per source box) of levels 2..L of `tree`, an oracle build
    of the source set against itself with lists; `owner` gives the node of
    every source box of level `lpar`."""
    L = tree["L"]
    if not 2 <= lpar <= L:
        raise ValueError("the partition level must be in 2..L")
    src = tree["src"]
    owner = np.asarray(owner)
    lcrit = max(lpar - 1, 2)
    # on[l][b] for l >= lpar: the owner of the box's ancestor at lpar is J
    on = {lpar: owner == node}
    for l in range(lpar + 1, L + 1):
        on[l] = on[l - 1][src["parent"][l].astype(np.int64)]
    # children on / off J of the boxes of lcrit (their descendants at lpar)
    if lcrit == lpar:
        child_on, child_off = on[lpar], ~on[lpar]
    else:
        ch = src["child"][lcrit].astype(np.int64)
        nb = len(src["key"][lcrit])
        child_on = np.array([bool(on[lpar][ch[k]:ch[k + 1]].any()) for k in range(nb)], bool)
        child_off = np.array([bool((~on[lpar][ch[k]:ch[k + 1]]).any()) for k in range(nb)], bool)
    out = {}
    for l in range(2, L + 1):
        nb = len(src["key"][l])
        t = np.full(nb, DOMESTIC, np.uint8)
        if l >= lcrit:
            e4o = tree["e4_off"][l].astype(np.int64)
            e4i = tree["e4_idx"][l].astype(np.int64)
            for k in range(nb):
                nbr = e4i[e4o[k]:e4o[k + 1]]
                if l == lcrit:
                    is_on_node, is_import_export = child_on[k], child_off[k]
                    if not is_on_node:
                        t[k] = IMPORT
                    elif is_import_export:
                        t[k] = ROOT
                    elif child_off[nbr].any():
                        t[k] = EXPORT
                else:
                    if not on[l][k]:
                        t[k] = IMPORT if on[l][nbr].any() else OTHERS
                    elif (~on[l][nbr]).any():
                        t[k] = EXPORT
        out[l] = t
    return out

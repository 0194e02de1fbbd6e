"""Word lists for the synthetic scan-record templates.

Written for this project: generic English and systems vocabulary of the kind a
vulnerability-scanner finding contains (service names, verbs, severities,
remediation phrasing). No scanner output, advisory text or CVE record is
reproduced here; the words are assembled into sentences at random.
"""

SERVICES = (
    "apache nginx tomcat openssh proftpd bind openldap mysql postgresql mongodb redis "
    "elasticsearch prometheus grafana jenkins gitlab nexus kafka rabbitmq zookeeper "
    "samba postfix dovecot exim squid haproxy varnish lighttpd memcached cassandra "
    "couchdb influxdb kibana logstash consul vault docker kubelet etcd containerd "
    "wordpress drupal joomla phpmyadmin webmin cups snmpd ntpd dnsmasq openvpn "
    "strongswan iis exchange sharepoint jboss wildfly weblogic websphere glassfish"
).split()

NOUNS = (
    "server service host port protocol version vulnerability certificate cipher "
    "configuration module plugin package library kernel daemon interface address "
    "network request response header cookie session token password credential "
    "account user administrator privilege permission directory file path endpoint "
    "parameter query buffer overflow injection traversal disclosure exposure "
    "component installation update patch release advisory vendor product platform "
    "system process memory stack heap pointer function method handler parser "
    "encoder decoder protocol handshake connection socket listener proxy gateway "
    "firewall router switch controller instance cluster node replica backup "
    "database table record schema index cache queue topic channel message "
    "signature algorithm hash key length strength expiry chain authority "
    "banner fingerprint timestamp scan result finding evidence output detail "
    "risk severity impact score vector solution workaround mitigation reference "
    "attacker adversary client browser application framework runtime container "
    "image volume secret policy rule filter mapping template report summary"
).split()

VERBS = (
    "allows enables permits exposes discloses reveals accepts supports uses "
    "contains includes returns sends receives reads writes executes runs "
    "listens responds fails validates checks verifies parses handles processes "
    "upgrade update install remove disable enable restrict configure apply "
    "detected identified reported observed found determined confirmed "
    "affects impacts crashes leaks bypasses escalates overwrites injects"
).split()

ADJECTIVES = (
    "remote local unauthenticated authenticated anonymous default weak strong "
    "outdated obsolete deprecated vulnerable insecure unsupported expired "
    "selfsigned untrusted invalid crafted malicious arbitrary sensitive internal "
    "external public private critical high medium low informational multiple "
    "several certain specific affected fixed later earlier current recent "
    "legacy minor major unknown known potential possible successful"
).split()

FUNCTION_WORDS = (
    "the a an of to in on at by for with from via and or not is are was be "
    "this that these those it its which when if than then as into over under "
    "before after all any each no may can could should would must has have "
    "version versions prior through up"
).split()

SEVERITIES = ("Critical", "High", "Medium", "Low", "Info")

PROTOCOLS = ("tcp", "udp")

TLDS = ("com", "net", "org", "local", "internal", "lan", "corp", "br", "edu", "io",
        "gov", "info", "cloud", "site")

HOST_WORDS = (
    "web srv db mail app api vpn proxy dc files backup build ci git wiki intranet "
    "portal auth sso ldap dns ntp mon log grafana kafka redis cache edge lb node "
    "worker gw fw core lab test dev stage prod campus noc soc ops"
).split()

ORG_WORDS = (
    "campus backbone datacenter research lab faculty institute network services "
    "library clinic office branch regional central north south east west"
).split()

FIELD_LABELS = (
    "Host", "Port", "Protocol", "Plugin", "Name", "Severity", "Risk", "Description",
    "Solution", "Synopsis", "Output", "Family", "Hostname", "Address", "Service",
    "Reference", "Evidence", "Detail", "Summary", "Impact",
)
